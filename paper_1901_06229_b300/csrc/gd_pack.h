// Host-side validation and packing of one ligand, shared by gd_dock_batch (gd_api.cu) and
// gd_dock_batch_noalloc (gd_noalloc.cu) so that both reject the same inputs with the same
// message and pack bit-identical inputs for the search kernel.  Not part of the public ABI.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>

#include "geodock.h"
#include "gd_internal.h"

namespace gd {

// printf-style failure report: records the message for the caller and returns the status.
typedef gd_status (*FailFn)(gd_status, const char*, ...);

// Validate ligand li (n atoms at xyz, nb bonds, R rotamer bonds) and write its atoms in DFS
// preorder from atom 0 (so the subtree under either end of a tree bond is one contiguous
// range), the preorder -> input permutation and one RotDesc per rotamer.  The rotamer's
// moving x static pairs closer than min_sep bonds are appended to excl[*n_excl ..] (at
// most excl_cap entries in all) as (a | b << 8), sorted by (a, b), and the descriptor
// records their offset and count.  cost (optional): an estimate of the ligand's search
// work, used to order the work queue.  Every temporary is a fixed-size array (n <=
// GD_MAX_ATOMS): no heap traffic, so many host threads can pack at once, and callers that
// must not allocate can use it.
inline gd_status pack_ligand_fixed(FailFn fail, int li, int n, const float* xyz, int nb, const int32_t* bonds, int R,
                                   const int32_t* rot_bond, int min_sep, float4* out_xyz, uint8_t* out_perm,
                                   RotDesc* out_rots, uint16_t* excl, size_t excl_cap, size_t* n_excl,
                                   double* cost) {
  if (n < 2 || n > GD_MAX_ATOMS) return fail(GD_EINVAL, "ligand %d: %d atoms outside [2, %d]", li, n, GD_MAX_ATOMS);
  if (nb != n - 1) return fail(GD_EINVAL, "ligand %d: %d bonds for %d atoms (not a tree)", li, nb, n);
  if (R < 0 || R > GD_MAX_ROTAMERS) return fail(GD_EINVAL, "ligand %d: %d rotamers > %d", li, R, GD_MAX_ROTAMERS);
  for (int i = 0; i < 3 * n; ++i)
    if (!std::isfinite(xyz[i])) return fail(GD_EINVAL, "ligand %d: non-finite coordinate", li);
  constexpr int NA = GD_MAX_ATOMS;
  int adj_off[NA + 1], adj[2 * NA], fill[NA];
  for (int i = 0; i <= n; ++i) adj_off[i] = 0;
  for (int b = 0; b < nb; ++b) {
    int u = bonds[2 * b], v = bonds[2 * b + 1];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v) return fail(GD_EINVAL, "ligand %d: bad bond %d", li, b);
    adj_off[u + 1]++;
    adj_off[v + 1]++;
  }
  for (int i = 0; i < n; ++i) {
    adj_off[i + 1] += adj_off[i];
    fill[i] = adj_off[i];
  }
  for (int b = 0; b < nb; ++b) {
    int u = bonds[2 * b], v = bonds[2 * b + 1];
    adj[fill[u]++] = v;
    adj[fill[v]++] = u;
  }
  // DFS preorder from atom 0; subtrees become contiguous ranges
  int parent[NA], pre[NA], order[NA], stack[2 * NA], size[NA];
  for (int i = 0; i < n; ++i) {
    parent[i] = -2;
    pre[i] = -1;
  }
  int n_order = 0, top = 0;
  stack[top++] = 0;
  parent[0] = -1;
  while (top) {
    int v = stack[--top];
    if (pre[v] >= 0) return fail(GD_EINVAL, "ligand %d: bonds contain a cycle (not a tree)", li);
    pre[v] = n_order;
    order[n_order++] = v;
    for (int e = adj_off[v + 1] - 1; e >= adj_off[v]; --e) {
      int w = adj[e];
      if (w == parent[v]) continue;
      if (pre[w] >= 0 || top >= 2 * NA) return fail(GD_EINVAL, "ligand %d: bonds contain a cycle (not a tree)", li);
      parent[w] = v;
      stack[top++] = w;
    }
  }
  if (n_order != n) return fail(GD_EINVAL, "ligand %d: bond graph is not connected", li);
  for (int i = 0; i < n; ++i) size[i] = 1;
  for (int t = n - 1; t > 0; --t) size[parent[order[t]]] += size[order[t]];
  for (int t = 0; t < n; ++t) {
    int v = order[t];
    out_xyz[t] = make_float4(xyz[3 * v], xyz[3 * v + 1], xyz[3 * v + 2], 0.f);
    out_perm[t] = (uint8_t)v;
  }
  double c = n;
  int depth[NA], queue[NA], near_m[NA], near_s[NA];
  uint16_t ex[GD_MAX_EXCLUDED];
  for (int r = 0; r < R; ++r) {
    const int b = rot_bond[r];
    if (b < 0 || b >= nb) return fail(GD_EINVAL, "ligand %d: rotamer %d names bond %d of %d", li, r, b, nb);
    int u = bonds[2 * b], v = bonds[2 * b + 1];
    int child = parent[v] == u ? v : u;
    int sub = size[child], rest = n - sub;
    if (sub == 1 || rest == 1) return fail(GD_EINVAL, "ligand %d: rotamer %d is on a terminal bond", li, r);
    RotDesc d{};
    d.comp = sub > rest ? 1 : 0;  // equal sides: move the subtree (the side without atom 0)
    int q = d.comp ? parent[child] : child;
    int p = d.comp ? child : parent[child];
    d.p = (uint16_t)pre[p];
    d.q = (uint16_t)pre[q];
    d.lo = (uint16_t)pre[child];
    d.hi = (uint16_t)(pre[child] + sub);
    auto moving = [&](int atom) {
      bool in = pre[atom] >= d.lo && pre[atom] < d.hi;
      return d.comp ? !in : in;
    };
    // atoms within min_sep-2 bonds of q (moving side) and of p (static side)
    for (int i = 0; i < n; ++i) depth[i] = -1;
    int nm = 0, ns = 0;
    for (int side = 0; side < 2; ++side) {
      int root = side ? p : q, qh = 0, qt = 0;
      queue[qt++] = root;
      depth[root] = 0;
      while (qh < qt) {
        int a = queue[qh++];
        if (side) near_s[ns++] = a;
        else near_m[nm++] = a;
        if (depth[a] >= min_sep - 2) continue;
        for (int e = adj_off[a]; e < adj_off[a + 1]; ++e) {
          int w = adj[e];
          if (depth[w] >= 0 || moving(w) != (side == 0)) continue;
          depth[w] = depth[a] + 1;
          queue[qt++] = w;
        }
      }
    }
    int ne = 0;
    for (int x = 0; x < nm; ++x)
      for (int y = 0; y < ns; ++y)
        if (depth[near_m[x]] + depth[near_s[y]] + 1 < min_sep) ++ne;
    if (ne > GD_MAX_EXCLUDED)
      return fail(GD_EINVAL, "ligand %d: rotamer %d has %d excluded pairs > %d", li, r, ne, GD_MAX_EXCLUDED);
    ne = 0;
    for (int x = 0; x < nm; ++x)
      for (int y = 0; y < ns; ++y)
        if (depth[near_m[x]] + depth[near_s[y]] + 1 < min_sep)
          ex[ne++] = (uint16_t)((pre[near_m[x]] << 8) | pre[near_s[y]]);  // sort key (a, b)
    std::sort(ex, ex + ne);
    for (int e = 0, run = 0; e < ne; ++e) {
      run = (e && (ex[e] >> 8) == (ex[e - 1] >> 8)) ? run + 1 : 1;
      if (run > GD_MAX_EXCLUDED_ATOM)
        return fail(GD_EINVAL, "ligand %d: rotamer %d has more than %d excluded pairs on one atom", li, r,
                    GD_MAX_EXCLUDED_ATOM);
    }
    if (*n_excl + (size_t)ne > excl_cap) return fail(GD_EINVAL, "ligand %d: excluded-pair table full", li);
    d.n_excl = (uint8_t)ne;
    d.excl_off = (uint32_t)*n_excl;
    for (int e = 0; e < ne; ++e) excl[(*n_excl)++] = (uint16_t)((ex[e] >> 8) | ((ex[e] & 0xFF) << 8));  // a | b << 8
    out_rots[r] = d;
    const int f = d.comp ? rest : sub;
    c += (double)f * (n - f) + 4.0 * f;
  }
  if (cost) *cost = c * (R > 0 ? 1.0 : 0.1);
  return GD_OK;
}

// Range checks of the search parameters (gd_dock_batch, gd_check_batch, gd_autotune and
// gd_dock_batch_noalloc).
inline gd_status check_params_fixed(FailFn fail, const gd_search_params* p) {
  if (!p) return fail(GD_EINVAL, "params is NULL");
  if (p->n_alpha < 1 || p->n_beta < 1 || p->n_gamma < 1)
    return fail(GD_EINVAL, "Euler grid sizes must be >= 1");
  const long long O = (long long)p->n_alpha * p->n_beta * p->n_gamma;
  if (O > GD_MAX_ORIENT) return fail(GD_EINVAL, "%lld orientations > %d", O, GD_MAX_ORIENT);
  if (p->n_angles < 1 || p->n_angles > GD_MAX_ANGLES)
    return fail(GD_EINVAL, "n_angles %d outside [1, %d]", p->n_angles, GD_MAX_ANGLES);
  if (!(p->bump_dist > 0.f) || !std::isfinite(p->bump_dist)) return fail(GD_EINVAL, "bump_dist must be > 0");
  if (p->min_bond_sep < 1 || p->min_bond_sep > 8) return fail(GD_EINVAL, "min_bond_sep outside [1, 8]");
  if (p->repetitions < 1 || p->repetitions > GD_MAX_REPS)
    return fail(GD_EINVAL, "repetitions outside [1, %d]", GD_MAX_REPS);
  if (p->tile < -1 || p->tile > gd::tile_count()) return fail(GD_EINVAL, "tile %d out of range", p->tile);
  if (p->rigid_span < 0 || p->rigid_span > 3) return fail(GD_EINVAL, "rigid_span outside [0, 3]");
  if (p->rigid_span > 0 && (!(p->rigid_step > 0.f) || !std::isfinite(p->rigid_step)))
    return fail(GD_EINVAL, "rigid_step must be > 0");
  return GD_OK;
}

}  // namespace gd
