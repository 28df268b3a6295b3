"""Python binding of libgeodock (include/geodock.h): argument marshalling only.

Every step of the pose search runs in the CUDA library; this module converts numpy
arrays to the C structs, passes CUDA stream handles (torch streams or raw handles)
and turns status codes into exceptions.  If the library has not been built, loading
fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import weakref
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeodock.so")

GD_OK, GD_EINVAL, GD_ENOMEM, GD_EBUDGET, GD_ECUDA, GD_ETIMEOUT, GD_EBUSY, GD_ENOTREADY = range(8)
GD_FLAG_DEBUG = 1
GD_FLAG_DEBUG_BUMPS = 2
GD_FLAG_NO_FILTER = 4
GD_FLAG_MASK_SWEEP = 8
GD_FLAG_TEST_STAGE_TIMEOUT = 16
STATUS_NAMES = {0: "GD_OK", 1: "GD_EINVAL", 2: "GD_ENOMEM", 3: "GD_EBUDGET", 4: "GD_ECUDA",
                5: "GD_ETIMEOUT", 6: "GD_EBUSY", 7: "GD_ENOTREADY"}

# every entry point declared in include/geodock.h
EXPORTS = ["gd_create", "gd_destroy", "gd_last_error", "gd_load_pocket", "gd_free_pocket",
           "gd_dock_batch", "gd_fetch_results", "gd_job_launch", "gd_job_download", "gd_job_bytes", "gd_job_free",
           "gd_check_batch", "gd_tile_count", "gd_tile_info", "gd_autotune", "gd_dock_batch_noalloc",
           "gd_prepare_batch", "gd_prepare_batch_sel", "gd_measure_peaks", "gd_job_info",
           "gd_server_create", "gd_server_submit", "gd_server_poll", "gd_server_collect", "gd_server_stats",
           "gd_server_test_hold", "gd_server_destroy", "gd_server_submit_restarts", "gd_server_reserve_sms"]


class GeoDockError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# Pointer fields are c_void_p filled with plain addresses (the C side sees the same
# pointers): building a typed ctypes pointer per array costs more than the search of a
# single ligand.
class LigandBatchC(C.Structure):
    _fields_ = [("n_ligands", C.c_int32), ("atom_off", C.c_void_p), ("xyz", C.c_void_p),
                ("bond_off", C.c_void_p), ("bonds", C.c_void_p), ("rot_off", C.c_void_p), ("rot_bond", C.c_void_p)]


class SearchParamsC(C.Structure):
    _fields_ = [("n_alpha", C.c_int32), ("n_beta", C.c_int32), ("n_gamma", C.c_int32),
                ("n_angles", C.c_int32), ("bump_dist", C.c_float), ("min_bond_sep", C.c_int32),
                ("repetitions", C.c_int32), ("flags", C.c_int32), ("tile", C.c_int32),
                ("rigid_span", C.c_int32), ("rigid_step", C.c_float)]


RESULT_FIELDS = ("best_score", "best_orient", "best_angle", "best_xyz", "evals", "pair_tests", "atom_moves",
                 "reach_tests", "orient_score", "orient_pick", "bump_bits", "best_rigid", "orient_rigid")


class ResultBatchC(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in RESULT_FIELDS]


_lib = None


def load():
    """Load libgeodock.so; raises if it is missing (build it with build.py / build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgeodock.so not found at {LIB_PATH}: build the CUDA library first "
                           "(python -m paper_1901_06229_b300.build)")
    L = C.CDLL(LIB_PATH)
    vp, P = C.c_void_p, C.POINTER
    L.gd_create.argtypes = [P(vp), C.c_int, C.c_size_t]
    L.gd_destroy.argtypes = [vp]
    L.gd_last_error.argtypes = [vp]
    L.gd_last_error.restype = C.c_char_p
    L.gd_load_pocket.argtypes = [vp, P(C.c_uint8), C.c_int, C.c_int, C.c_int, C.c_float, P(C.c_float), P(vp)]
    L.gd_free_pocket.argtypes = [vp, vp]
    L.gd_dock_batch.argtypes = [vp, vp, P(LigandBatchC), P(SearchParamsC), vp, P(vp)]
    L.gd_fetch_results.argtypes = [vp, vp, P(ResultBatchC), C.c_int]
    L.gd_job_launch.argtypes = [vp, vp, vp]
    L.gd_job_download.argtypes = [vp, vp, vp]
    L.gd_job_free.argtypes = [vp, vp]
    L.gd_job_bytes.argtypes = [vp, vp, P(C.c_uint64), P(C.c_uint64)]
    L.gd_job_info.argtypes = [vp, vp, P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_int), P(C.c_size_t)]
    L.gd_server_create.argtypes = [vp, vp, P(SearchParamsC), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P(vp)]
    L.gd_server_submit.argtypes = [vp, P(LigandBatchC), vp, C.c_int32, P(C.c_uint64)]
    L.gd_server_poll.argtypes = [vp, C.c_uint64, P(ResultBatchC), C.c_int]
    L.gd_server_collect.argtypes = [vp, vp, vp, vp, C.c_int, P(C.c_int)]
    L.gd_server_stats.argtypes = [vp] + [P(C.c_uint64)] * 6
    L.gd_server_test_hold.argtypes = [vp, C.c_int64]
    L.gd_server_submit_restarts.argtypes = [vp, P(LigandBatchC), vp, C.c_int32, vp, vp, C.c_int32, P(C.c_uint64)]
    L.gd_server_reserve_sms.argtypes = [vp, C.c_int]
    L.gd_server_destroy.argtypes = [vp]
    L.gd_check_batch.argtypes = [P(LigandBatchC), P(SearchParamsC)]
    L.gd_prepare_batch.argtypes = [vp, vp, P(LigandBatchC), P(SearchParamsC), vp, P(vp)]
    L.gd_prepare_batch_sel.argtypes = [vp, vp, P(LigandBatchC), P(C.c_int32), C.c_int32, P(SearchParamsC), vp,
                                       P(vp)]
    L.gd_job_features.argtypes = [vp, vp, vp, vp, vp]
    L.gd_job_features.restype = C.c_int
    L.gd_job_launch_proposed.argtypes = [vp, vp, vp, C.c_int, C.c_float, C.c_int, vp]
    L.gd_job_launch_proposed.restype = C.c_int
    L.gd_job_launch_proposed_fb.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_float, C.c_int, vp]
    L.gd_job_launch_proposed_fb.restype = C.c_int
    L.gd_job_selection.argtypes = [vp, vp, vp, vp]
    L.gd_job_selection.restype = C.c_int
    L.gd_tile_count.argtypes = []
    L.gd_tile_info.argtypes = [C.c_int, P(C.c_int), P(C.c_int), P(C.c_int)]
    L.gd_autotune.argtypes = [vp, vp, P(LigandBatchC), P(SearchParamsC), C.c_int, vp, P(C.c_int), P(C.c_float)]
    for f in EXPORTS:
        if f not in ("gd_last_error",):
            getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _addr(a):
    """Address of a numpy array's first element."""
    return a.ctypes.data


class Results(dict):
    """Result arrays by name (see gd_result_batch); .addrs holds their addresses."""
    addrs = None


def result_arrays(L, N, Rt, reps, O, A, debug=False, bumps=False, rigid=True):
    """Host arrays of one result batch (gd_result_batch), views of one buffer; with debug
    the per-restart arrays, with bumps the per-candidate bump bits.  Every element is
    written by gd_fetch_results."""
    key = (L, N, Rt, reps, O, A, debug, bumps, rigid)
    lay = _LAYOUTS.get(key)
    if lay is None:
        spec = [("best_score", _U32, L, None), ("best_orient", _I32, L, None), ("best_angle", _I16, Rt * reps, None),
                ("best_xyz", _F32, 3 * N, (N, 3)), ("evals", _U64, L, None), ("pair_tests", _U64, L, None),
                ("atom_moves", _U64, L, None), ("reach_tests", _U64, L, None)]
        if rigid:
            spec.append(("best_rigid", _I16, L, None))
        if debug:
            spec += [("orient_score", _U32, L * O, (L, O)), ("orient_pick", _I16, Rt * reps * O, None),
                     ("orient_rigid", _I16, L * O, (L, O))]
        if bumps:
            spec.append(("bump_bits", _U8, Rt * reps * O * A, None))
        rows, o = [], 0
        for name, t, n, shape in spec:
            rows.append((name, t, o, o + n * t.itemsize, shape))
            o = (o + n * t.itemsize + 15) & ~15
        lay = (rows, max(o, 16))
        if len(_LAYOUTS) > 64:
            _LAYOUTS.clear()
        _LAYOUTS[key] = lay
    rows, total = lay
    buf = np.empty(total, np.uint8)
    base = buf.ctypes.data
    out = Results()
    addrs = out.addrs = {}
    for name, t, o0, o1, shape in rows:
        a = buf[o0:o1].view(t)
        out[name] = a if shape is None else a.reshape(shape)
        addrs[name] = base + o0
    return out


_LAYOUTS = {}
_U8, _I16, _I32, _U32, _U64, _F32 = (np.dtype(t) for t in (np.uint8, np.int16, np.int32, np.uint32, np.uint64,
                                                            np.float32))


def result_c(r):
    """gd_result_batch pointing at the arrays of r (NULL for absent ones)."""
    addrs = getattr(r, "addrs", None)
    if addrs is None:  # a caller's own dict of arrays
        for name in RESULT_FIELDS:
            if name in r and not r[name].flags.c_contiguous:
                raise ValueError(f"result array {name} must be C-contiguous")
        addrs = {name: _addr(r[name]) for name in RESULT_FIELDS if name in r}
    return ResultBatchC(*(addrs.get(name) for name in RESULT_FIELDS))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def params_c(params, flags=0, tile=0) -> SearchParamsC:
    return SearchParamsC(params.n_alpha, params.n_beta, params.n_gamma, params.n_angles,
                         float(params.bump_dist), params.min_bond_sep, params.repetitions, flags, tile,
                         int(getattr(params, "rigid_span", 0)), float(getattr(params, "rigid_step", 0.0)))


class _BatchArrays:
    """Keeps the contiguous numpy arrays alive while C holds pointers to them.  When the
    batch's arrays are already contiguous in the right types they are used in place, and
    the view is kept on the batch for the next call while its arrays are the same objects
    (the library reads their contents at every call)."""

    _TYPES = (("atom_off", np.int32), ("xyz", np.float32), ("bond_off", np.int32), ("bonds", np.int32),
              ("rot_off", np.int32), ("rot_bond", np.int32))

    def __new__(cls, batch):
        src = tuple(getattr(batch, name) for name, _ in cls._TYPES)
        cached = getattr(batch, "_gd_arrays", None)
        if cached is not None and all(a is b for a, b in zip(cached._src, src)):
            return cached
        self = super().__new__(cls)
        arrs = [np.ascontiguousarray(a, t) for a, (_, t) in zip(src, cls._TYPES)]
        for (name, _), a in zip(cls._TYPES, arrs):
            setattr(self, name, a)
        self._src = src
        self.c = LigandBatchC(len(self.atom_off) - 1, *(_addr(a) for a in arrs))
        if all(a is b for a, b in zip(arrs, src)):  # in place: safe to reuse while the arrays stay
            try:
                batch._gd_arrays = self
            except AttributeError:
                pass
        return self


class Job:
    def __init__(self, ctx, handle, batch, params, debug, bumps=False, sel=None):
        self.ctx, self.handle, self.debug, self.bumps = ctx, handle, debug or bumps, bumps
        if sel is None:
            self.L = batch.n_ligands
            self.N = len(batch.xyz)
            self.rot_off = np.asarray(batch.rot_off, np.int64)
        else:  # the job holds ligands sel of batch, packed in that order
            self.L = len(sel)
            self.N = int(np.diff(batch.atom_off)[sel].sum())
            self.rot_off = np.concatenate([[0], np.cumsum(np.diff(batch.rot_off)[sel])]).astype(np.int64)
        self.params = params

    def fetch(self, blocking=True, out=None):
        """Results as numpy arrays (see gd_result_batch); None if not ready (non-blocking)."""
        p = self.params
        O, reps, A = p.n_alpha * p.n_beta * p.n_gamma, p.repetitions, p.n_angles
        Rt = int(self.rot_off[-1]) if len(self.rot_off) else 0
        r = out if out is not None else result_arrays(self.L, self.N, Rt, reps, O, A, self.debug, self.bumps)
        st = load().gd_fetch_results(self.ctx.h, self.handle, C.byref(result_c(r)), 1 if blocking else 0)
        if st == GD_ENOTREADY:
            return None
        self.ctx._check(st)
        return r

    def features(self, x_bf16=None, x_f32=None, stream=None):
        """gd_job_features into torch CUDA tensors [L*O, 48] (BF16 and/or FP32)."""
        p = lambda t: C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)
        self.ctx._check(load().gd_job_features(self.ctx.h, self.handle, p(x_bf16), p(x_f32), _stream_handle(stream)))

    def launch_proposed(self, pred, k, margin, rule=1, stream=None, k_fallback=None):
        """gd_job_launch_proposed(_fb): search the k best-predicted restarts per ligand, the
        k_fallback best (all of them when None) where the top-k spread is below (rule 0) /
        above (rule 1) margin; pred is a CUDA float tensor [L*O]."""
        if k_fallback is None:
            self.ctx._check(load().gd_job_launch_proposed(self.ctx.h, self.handle, C.c_void_p(pred.data_ptr()),
                                                          int(k), float(margin), int(rule), _stream_handle(stream)))
        else:
            self.ctx._check(load().gd_job_launch_proposed_fb(self.ctx.h, self.handle, C.c_void_p(pred.data_ptr()),
                                                             int(k), int(k_fallback), float(margin), int(rule),
                                                             _stream_handle(stream)))

    def selection(self):
        """(restarts searched per ligand, prediction spread per ligand) of the last proposed launch."""
        cnt = np.zeros(self.L, np.int32)
        spr = np.zeros(self.L, np.float32)
        self.ctx._check(load().gd_job_selection(self.ctx.h, self.handle, C.c_void_p(cnt.ctypes.data),
                                                C.c_void_p(spr.ctypes.data)))
        return cnt, spr

    def launch(self, stream=None):
        """Run the search again on the device-resident inputs (no host copies)."""
        self.ctx._check(load().gd_job_launch(self.ctx.h, self.handle, _stream_handle(stream)))

    def download(self, stream=None):
        self.ctx._check(load().gd_job_download(self.ctx.h, self.handle, _stream_handle(stream)))

    def bytes_moved(self):
        """(host->device, device->host) bytes of one gd_dock_batch of this job."""
        i, o = C.c_uint64(), C.c_uint64()
        self.ctx._check(load().gd_job_bytes(self.ctx.h, self.handle, C.byref(i), C.byref(o)))
        return i.value, o.value

    def info(self):
        """gd_job_info: the search launch's tile, grid staging mode and shape."""
        t, g, b, th, sm = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_size_t()
        self.ctx._check(load().gd_job_info(self.ctx.h, self.handle, C.byref(t), C.byref(g), C.byref(b), C.byref(th),
                                           C.byref(sm)))
        return dict(tile=t.value, grid_in_smem=bool(g.value), blocks=b.value, threads=th.value, smem=sm.value)

    def free(self):
        if self.handle:
            load().gd_job_free(self.ctx.h, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Pocket:
    def __init__(self, ctx, handle):
        self.ctx, self.handle = ctx, handle
        self._servers = weakref.WeakSet()  # servers searching this pocket: closed before it is freed

    def free(self):
        if self.handle:
            for srv in list(self._servers):
                srv.close()
            if self.ctx.h:
                load().gd_free_pocket(self.ctx.h, self.handle)
            self.handle = None


class Context:
    """A gd_ctx on one CUDA device."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        L = load()
        h = C.c_void_p()
        st = L.gd_create(C.byref(h), int(device), C.c_size_t(mem_budget_bytes))
        if st:
            raise GeoDockError(st, L.gd_last_error(None).decode())
        self.h = h
        self._servers = weakref.WeakSet()  # closed before the context is

    def _check(self, st):
        if st:
            raise GeoDockError(st, load().gd_last_error(self.h).decode())

    def close(self):
        if self.h:
            for srv in list(self._servers):
                srv.close()
            load().gd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load_pocket(self, pocket) -> Pocket:
        g = np.ascontiguousarray(pocket.grid, np.uint8)
        nz, ny, nx = g.shape
        org = np.ascontiguousarray(pocket.origin, np.float32)
        h = C.c_void_p()
        self._check(load().gd_load_pocket(self.h, _ptr(g, C.c_uint8), nx, ny, nz, float(pocket.spacing),
                                          _ptr(org, C.c_float), C.byref(h)))
        return Pocket(self, h)

    def dock_batch(self, pocket: Pocket, batch, params, stream=None, debug=False, bumps=False, tile=0,
                   no_filter=False, mask_sweep=False, test_stage_timeout=False) -> Job:
        """gd_dock_batch: debug keeps per-restart scores/picks, bumps also per-candidate bump bits,
        no_filter tests every pair at every angle, mask_sweep sweeps the reach filter's bit masks
        instead of its near list (same results either way); test_stage_timeout makes the
        grid-staging wait run out (testing the device-timeout report)."""
        arrs = _BatchArrays(batch)
        flags = ((GD_FLAG_DEBUG if debug else 0) | (GD_FLAG_DEBUG_BUMPS if bumps else 0)
                 | (GD_FLAG_NO_FILTER if no_filter else 0) | (GD_FLAG_MASK_SWEEP if mask_sweep else 0)
                 | (GD_FLAG_TEST_STAGE_TIMEOUT if test_stage_timeout else 0))
        prm = params_c(params, flags, tile)
        h = C.c_void_p()
        self._check(load().gd_dock_batch(self.h, pocket.handle, C.byref(arrs.c), C.byref(prm),
                                         _stream_handle(stream), C.byref(h)))
        return Job(self, h, batch, params, debug, bumps)

    def prepare_batch(self, pocket: Pocket, batch, params, stream=None, debug=False, tile=0, sel=None) -> Job:
        """gd_prepare_batch: validate, pack and upload without searching; with sel (ligand
        indices into batch), gd_prepare_batch_sel: the job holds those ligands in that order."""
        arrs = _BatchArrays(batch)
        prm = params_c(params, GD_FLAG_DEBUG if debug else 0, tile)
        h = C.c_void_p()
        if sel is None:
            self._check(load().gd_prepare_batch(self.h, pocket.handle, C.byref(arrs.c), C.byref(prm),
                                                _stream_handle(stream), C.byref(h)))
        else:
            sel = np.ascontiguousarray(sel, np.int32)
            self._check(load().gd_prepare_batch_sel(self.h, pocket.handle, C.byref(arrs.c), _ptr(sel, C.c_int32),
                                                    len(sel), C.byref(prm), _stream_handle(stream), C.byref(h)))
        return Job(self, h, batch, params, debug, sel=sel)

    def autotune(self, pocket: Pocket, batch, params, max_ligands=256, stream=None, no_filter=False):
        arrs = _BatchArrays(batch)
        prm = params_c(params, GD_FLAG_NO_FILTER if no_filter else 0)
        t, ms = C.c_int(), C.c_float()
        self._check(load().gd_autotune(self.h, pocket.handle, C.byref(arrs.c), C.byref(prm), int(max_ligands),
                                       _stream_handle(stream), C.byref(t), C.byref(ms)))
        return t.value, ms.value


class Server:
    """gd_server: ligands submitted over time join one running search launch (continuous
    batching on the device); results come back per ligand, numbered in submission order.
    The pocket must stay loaded while the server exists."""

    def __init__(self, ctx, pocket, params, capacity=4096, max_atoms=256, max_rotamers=64, max_excluded=0,
                 idle_ms=200, tile=0, free_sms=0):
        self.ctx, self.params = ctx, params
        self.h = None
        h = C.c_void_p()
        prm = params_c(params, 0, tile)
        ctx._check(load().gd_server_create(ctx.h, pocket.handle, C.byref(prm), int(capacity), int(max_atoms),
                                           int(max_rotamers), int(max_excluded), int(idle_ms), C.byref(h)))
        self.h = h
        ctx._servers.add(self)
        pocket._servers.add(self)
        if free_sms:  # gd_server_reserve_sms: SMs left to other kernels (before any submission)
            ctx._check(load().gd_server_reserve_sms(h, int(free_sms)))
        self.capacity = capacity
        self._sizes = {}  # seq -> (atoms, rotamers) of ligands not yet returned in full

    def submit(self, batch, sel=None, restarts=None, n_restarts=None) -> int:
        """Submit ligands sel of batch (all when None); returns the first sequence number
        (GeoDockError GD_EBUSY when there are not enough free slots).  With restarts (a
        [n, stride] array of restart ids) and n_restarts ([n]), ligand i searches only
        restarts[i, :n_restarts[i]] (gd_server_submit_restarts)."""
        arrs = _BatchArrays(batch)
        first = C.c_uint64()
        n = batch.n_ligands if sel is None else len(sel)
        selp = None
        if sel is not None:
            sel = np.ascontiguousarray(sel, np.int32)
            selp = C.c_void_p(_addr(sel))
        if restarts is None:
            self.ctx._check(load().gd_server_submit(self.h, C.byref(arrs.c), selp, n, C.byref(first)))
        else:
            res = np.ascontiguousarray(restarts, np.uint16)
            cnt = np.ascontiguousarray(n_restarts, np.int32)
            assert res.ndim == 2 and res.shape[0] == n and cnt.shape == (n,)
            self.ctx._check(load().gd_server_submit_restarts(self.h, C.byref(arrs.c), selp, n,
                                                             C.c_void_p(_addr(res)), C.c_void_p(_addr(cnt)),
                                                             int(res.shape[1]), C.byref(first)))
        idx = range(n) if sel is None else sel
        na, nr = np.diff(batch.atom_off), np.diff(batch.rot_off)
        for k, i in enumerate(idx):
            self._sizes[first.value + k] = (int(na[i]), int(nr[i]))
        return first.value

    def poll(self, seq, blocking=True):
        """Full results of ligand seq (one-ligand result arrays), or None if not ready."""
        n, R = self._sizes[seq]
        r = result_arrays(1, n, R, self.params.repetitions, 1, 1)
        st = load().gd_server_poll(self.h, int(seq), C.byref(result_c(r)), 1 if blocking else 0)
        if st == GD_ENOTREADY:
            return None
        self.ctx._check(st)
        del self._sizes[seq]
        return r

    def collect(self, max_n=4096):
        """(seqs, best scores, best restarts) of the finished ligands not returned yet."""
        seq = np.empty(max_n, np.uint64)
        sc = np.empty(max_n, np.uint32)
        ob = np.empty(max_n, np.int32)
        k = C.c_int()
        self.ctx._check(load().gd_server_collect(self.h, C.c_void_p(_addr(seq)), C.c_void_p(_addr(sc)),
                                                 C.c_void_p(_addr(ob)), int(max_n), C.byref(k)))
        n = k.value
        for q in seq[:n].tolist():
            self._sizes.pop(q, None)
        return seq[:n], sc[:n], ob[:n]

    def stats(self):
        v = [C.c_uint64() for _ in range(6)]
        self.ctx._check(load().gd_server_stats(self.h, *(C.byref(x) for x in v)))
        return dict(zip(("launches", "idle_exits", "published", "finished", "claimed_items", "control_reads"),
                        (x.value for x in v)))

    def test_hold(self, seq):
        """Testing only: the slot of ligand seq is never released on the device (-1: off)."""
        self.ctx._check(load().gd_server_test_hold(self.h, int(seq)))

    def close(self):
        """Destroy the server (before its context and pocket go; they close it otherwise)."""
        if self.h:
            if self.ctx.h:
                load().gd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_batch(batch, params) -> None:
    """gd_check_batch: host-only validation; raises GeoDockError(GD_EINVAL) with the reason."""
    arrs = _BatchArrays(batch)
    prm = params_c(params)
    st = load().gd_check_batch(C.byref(arrs.c), C.byref(prm))
    if st:
        raise GeoDockError(st, load().gd_last_error(None).decode())


def dock_noalloc(batch, pocket, params, stream=None, tile=0) -> dict:
    """gd_dock_batch_noalloc: dock without any allocation at call time (synchronous).

    For callers that cannot allocate device memory when they dock (device memory
    already reserved by another allocator, allocation forbidden after start-up, or
    cudaMalloc/cudaFree's device-wide synchronisation unacceptable): the library's
    fixed 64 MiB device array holds the grid, packed ligands, results and scratch.
    Calls share that array, so overlapping calls race.
    """
    L = load()
    if not hasattr(L, "_noalloc_ready"):
        L.gd_dock_batch_noalloc.argtypes = [C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int, C.c_float,
                                            C.POINTER(C.c_float), C.POINTER(LigandBatchC), C.POINTER(SearchParamsC),
                                            C.POINTER(ResultBatchC), C.c_void_p, C.c_char_p, C.c_size_t]
        L.gd_dock_batch_noalloc.restype = C.c_int
        L._noalloc_ready = True
    arrs = _BatchArrays(batch)
    prm = params_c(params, 0, tile)
    g = np.ascontiguousarray(pocket.grid, np.uint8)
    nz, ny, nx = g.shape
    org = np.ascontiguousarray(pocket.origin, np.float32)
    n_lig, n_atoms, Rt = batch.n_ligands, len(batch.xyz), int(batch.rot_off[-1]) if len(batch.rot_off) else 0
    r = result_arrays(n_lig, n_atoms, Rt, params.repetitions, params.n_orient, params.n_angles, rigid=False)
    rb = result_c(r)
    msg = C.create_string_buffer(512)
    st = L.gd_dock_batch_noalloc(_ptr(g, C.c_uint8), nx, ny, nz, float(pocket.spacing), _ptr(org, C.c_float),
                                 C.byref(arrs.c), C.byref(prm), C.byref(rb), _stream_handle(stream), msg, 512)
    if st:
        raise GeoDockError(st, msg.value.decode())
    return r


def tile_count() -> int:
    return load().gd_tile_count()


def tile_info(tile: int):
    """(warps per block, angles per lane, register budget per thread) of a tile id."""
    w, s, r = C.c_int(), C.c_int(), C.c_int()
    st = load().gd_tile_info(int(tile), C.byref(w), C.byref(s), C.byref(r))
    if st:
        raise GeoDockError(st, load().gd_last_error(None).decode())
    return w.value, s.value, r.value


def measure_peaks(device: int = 0, stream=None) -> dict:
    """Measured peaks of the search kernel's pipes on one device (gd_measure_peaks):
    FP32 FMAs per second and shared-memory byte loads per second, both per lane."""
    f, l = C.c_double(), C.c_double()
    st = load().gd_measure_peaks(int(device), _stream_handle(stream), C.byref(f), C.byref(l))
    if st:
        raise GeoDockError(st, load().gd_last_error(None).decode())
    return {"ffma_per_s": f.value, "lds_u8_per_s": l.value}


def dock(batch, pocket, params, device=0, debug=False, bumps=False, tile=0, stream=None) -> dict:
    """One-shot convenience: create a context, dock, fetch, clean up."""
    with Context(device) as ctx:
        pk = ctx.load_pocket(pocket)
        job = ctx.dock_batch(pk, batch, params, stream=stream, debug=debug, bumps=bumps, tile=tile)
        out = job.fetch(blocking=True)
        job.free()
        pk.free()
    return out
