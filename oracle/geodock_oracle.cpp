// GeoDock pose-search oracle: plain, slow, FP64, single-threaded per ligand.
//
// TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is checked
// against; only the test suite, the package smoke check and the CPU-baseline leg of
// the benchmark may load it.  It shares no code, header or table with the CUDA
// library and derives topology, fragments, placement and scores on its own.
//
// What it computes (the paper's GeoDock algorithm, Sec. 3.1, Listing 1):
//   for every ligand (independent, Sec. 1):
//     for every restart pose_id < N:          generate_starting_pose  (Listing 1)
//       place the ligand rigidly in the pocket  align_ligand (rigid phase, Sec. 3.1)
//       repeat num_repetitions times:           optimize_pose           (Sec. 3.1)
//         for every fragment, in sequence:      "each fragment is sequentially rotated"
//           rotate the fragment about its 1-D bond axis through a discrete angle
//           set (Sec. 4.1), reject bumped candidates (BumpCheck, Sec. 3.2), score
//           the rest (scoring function, Sec. 3.2), keep the best (reduction after
//           every fragment, Sec. 4.1)
//     keep the best-scoring restart (reduction over orientations, Sec. 4.1).
// The paper leaves the scoring function, bump rule, angle set, restart generator
// and grid unspecified; the readings implemented here are:
//   * restarts   = ZYZ Euler grid: alpha = 2 pi i / na, beta = pi (j + 1/2) / nb,
//                  gamma = 2 pi k / ng, o = (i nb + j) ng + k, R = Rz(a) Ry(b) Rz(g);
//                  x <- c_pocket + R (x - c_lig), c_lig = unweighted centroid,
//                  c_pocket = origin + h (nx, ny, nz) / 2.
//   * score      = sum over atoms of grid[floor((x - origin) / h)], 0 outside the box.
//   * fragment   = smaller side of the rotamer bond (tie: the side without atom 0);
//                  p = static endpoint, q = moving endpoint, axis u = (x_q - x_p)/|.|
//                  taken from the current coordinates.
//   * angles     = theta_k = 2 pi k / A, k in [0, A); right-handed about u (Rodrigues).
//   * bump       = some moving atom a and static atom b with graph distance >= min_sep
//                  and |x'_a - x_b| < bump_dist (strict).
//   * pick       = highest score among unbumped candidates, ties to the smallest k;
//                  if every candidate is bumped the pose is kept (recorded as -1).
//   * best pose  = highest final score over orientations, ties to the smallest o.
//
// Besides the values, the oracle marks *fragile* decisions: those a perturbation of
// the coordinates by eps (1e-4 A) could flip -- an atom within eps of a cell face
// whose neighbour cell has another value, or a pair within eps of bump_dist -- so that
// an FP32 implementation can be compared exactly everywhere else.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct M3 {
  double m[3][3];
};
inline V3 mul(const M3& R, V3 v) {
  return {R.m[0][0] * v.x + R.m[0][1] * v.y + R.m[0][2] * v.z,
          R.m[1][0] * v.x + R.m[1][1] * v.y + R.m[1][2] * v.z,
          R.m[2][0] * v.x + R.m[2][1] * v.y + R.m[2][2] * v.z};
}
inline M3 matmul(const M3& A, const M3& B) {
  M3 C{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) C.m[i][j] += A.m[i][k] * B.m[k][j];
  return C;
}
inline M3 rot_z(double t) {
  double c = std::cos(t), s = std::sin(t);
  return M3{{{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}}};
}
inline M3 rot_y(double t) {
  double c = std::cos(t), s = std::sin(t);
  return M3{{{c, 0.0, s}, {0.0, 1.0, 0.0}, {-s, 0.0, c}}};
}

// Restart orientation o of an (na, nb, ng) Euler grid (generate_starting_pose).
M3 euler_orientation(int o, int na, int nb, int ng) {
  const double pi = 3.14159265358979323846;
  int i = o / (nb * ng);
  int j = (o / ng) % nb;
  int k = o % ng;
  double alpha = 2.0 * pi * i / na;
  double beta = pi * (j + 0.5) / nb;
  double gamma = 2.0 * pi * k / ng;
  return matmul(matmul(rot_z(alpha), rot_y(beta)), rot_z(gamma));
}

// Rotation of v by theta about the unit axis u (Rodrigues' formula).
inline V3 rodrigues(V3 u, double theta, V3 v) {
  double c = std::cos(theta), s = std::sin(theta);
  return c * v + s * cross(u, v) + ((1.0 - c) * dot(u, v)) * u;
}

struct Pocket {
  const uint8_t* grid;
  int nx, ny, nz;
  double h;
  V3 origin;
};

// Centre of the grid box, where restarts place the ligand's centroid.
inline V3 pocket_centre(V3 origin, double h, int nx, int ny, int nz) {
  return origin + (0.5 * h) * V3{(double)nx, (double)ny, (double)nz};
}

// Cell value at x: grid[floor((x - origin)/h)], 0 outside the box (scoring function).
int cell_value(const Pocket& P, V3 x) {
  double u[3] = {(x.x - P.origin.x) / P.h, (x.y - P.origin.y) / P.h, (x.z - P.origin.z) / P.h};
  int n[3] = {P.nx, P.ny, P.nz};
  long idx[3];
  for (int d = 0; d < 3; ++d) {
    double f = std::floor(u[d]);
    if (!(f >= 0.0 && f < n[d])) return 0;
    idx[d] = (long)f;
  }
  return P.grid[(idx[2] * P.ny + idx[1]) * P.nx + idx[0]];
}

// Smallest and largest cell value any point within eps (per axis) of x can read.
void cell_range(const Pocket& P, V3 x, double eps, int* lo, int* hi) {
  double c[3] = {x.x, x.y, x.z};
  double alt[3][2];
  for (int d = 0; d < 3; ++d) {
    alt[d][0] = c[d] - eps;
    alt[d][1] = c[d] + eps;
  }
  int mn = 1 << 30, mx = -1;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int g = 0; g < 2; ++g) {
        int v = cell_value(P, V3{alt[0][a], alt[1][b], alt[2][g]});
        mn = std::min(mn, v);
        mx = std::max(mx, v);
      }
  int v0 = cell_value(P, x);
  *lo = std::min(mn, v0);
  *hi = std::max(mx, v0);
}

struct Params {
  int n_alpha, n_beta, n_gamma, n_angles;
  double bump_dist;
  int min_bond_sep;
  int repetitions;
  int rigid_span;     // rigid alignment sweep (align_ligand): (2s+1)^3 rotations, 0 = off
  double rigid_step;  // radians
};

// Rigid candidate m of the sweep: m = 0 is the identity, the others are the rotation
// vectors step * (i - s, j - s, k - s), i, j, k in [0, 2s], in (i, j, k) order without
// the zero vector; as a rotation about that vector's direction by its length.
M3 rigid_candidate(int m, int s, double step) {
  M3 I{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
  if (m == 0) return I;
  int count = 0;
  const int W = 2 * s + 1;
  for (int i = 0; i < W; ++i)
    for (int j = 0; j < W; ++j)
      for (int k = 0; k < W; ++k) {
        if (i == s && j == s && k == s) continue;
        if (++count != m) continue;
        const V3 v{step * (i - s), step * (j - s), step * (k - s)};
        const double th = norm(v);
        const V3 u = (1.0 / th) * v;
        M3 R{};
        const V3 ex{1, 0, 0}, ey{0, 1, 0}, ez{0, 0, 1};
        const V3 cx = rodrigues(u, th, ex), cy = rodrigues(u, th, ey), cz = rodrigues(u, th, ez);
        R.m[0][0] = cx.x; R.m[1][0] = cx.y; R.m[2][0] = cx.z;
        R.m[0][1] = cy.x; R.m[1][1] = cy.y; R.m[2][1] = cy.z;
        R.m[0][2] = cz.x; R.m[1][2] = cz.y; R.m[2][2] = cz.z;
        return R;
      }
  return I;
}

struct Topo {
  int n = 0;
  std::vector<std::vector<int>> adj;
  std::vector<int> dist;  // n*n graph distances (bonds)
};

struct Rotamer {
  int p = -1, q = -1;             // static / moving endpoint of the rotamer bond
  std::vector<char> moving;       // 1 for atoms of the rotating fragment
  std::vector<std::pair<int, int>> pairs;  // moving x static pairs with dist >= min_sep
};

bool build_topology(int n, const int32_t* bonds, int nb, Topo& t, std::string& err) {
  if (n < 2) { err = "fewer than 2 atoms"; return false; }
  if (nb != n - 1) { err = "bond count is not atoms-1 (not a tree)"; return false; }
  t.n = n;
  t.adj.assign(n, {});
  for (int b = 0; b < nb; ++b) {
    int u = bonds[2 * b], v = bonds[2 * b + 1];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v) { err = "bad bond"; return false; }
    t.adj[u].push_back(v);
    t.adj[v].push_back(u);
  }
  t.dist.assign((size_t)n * n, -1);
  for (int s = 0; s < n; ++s) {  // breadth-first search from every atom
    std::vector<int> queue{s};
    t.dist[(size_t)s * n + s] = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
      int a = queue[h];
      for (int b : t.adj[a])
        if (t.dist[(size_t)s * n + b] < 0) {
          t.dist[(size_t)s * n + b] = t.dist[(size_t)s * n + a] + 1;
          queue.push_back(b);
        }
    }
    if ((int)queue.size() != n) { err = "bond graph is not connected (not a tree)"; return false; }
  }
  return true;
}

bool build_rotamer(const Topo& t, const int32_t* bonds, int nb, int rb, int min_sep, Rotamer& r,
                   std::string& err) {
  if (rb < 0 || rb >= nb) { err = "rotamer bond index out of range"; return false; }
  int u = bonds[2 * rb], v = bonds[2 * rb + 1];
  const int n = t.n;
  // side of u once the bond u-v is cut
  std::vector<char> side_u(n, 0);
  std::vector<int> queue{u};
  side_u[u] = 1;
  for (size_t h = 0; h < queue.size(); ++h)
    for (int b : t.adj[queue[h]]) {
      if ((queue[h] == u && b == v) || side_u[b]) continue;
      side_u[b] = 1;
      queue.push_back(b);
    }
  int nu = (int)queue.size(), nv = n - nu;
  if (nu == 1 || nv == 1) { err = "rotamer on a terminal bond"; return false; }
  bool frag_is_v;
  if (nv != nu) frag_is_v = nv < nu;
  else frag_is_v = side_u[0] != 0;  // equal sides: move the side without atom 0
  r.q = frag_is_v ? v : u;
  r.p = frag_is_v ? u : v;
  r.moving.assign(n, 0);
  for (int a = 0; a < n; ++a) r.moving[a] = frag_is_v ? !side_u[a] : side_u[a];
  r.pairs.clear();
  for (int a = 0; a < n; ++a)
    if (r.moving[a])
      for (int b = 0; b < n; ++b)
        if (!r.moving[b] && t.dist[(size_t)a * n + b] >= min_sep) r.pairs.push_back({a, b});
  return true;
}

// BumpCheck's pair rule (Sec. 3.2): a pair bumps when strictly closer than bump_dist.
inline bool bumps(double d, double bump_dist) { return d < bump_dist; }

// Bump status of one candidate: 0 free, 1 bumped, 2 uncertain (a pair within eps of
// the threshold and no pair clearly inside it).  *first_bump is the position of the
// first pair closer than bump_dist in the list order (moving atom ascending, then
// static atom ascending), -1 if there is none.
int bump_status(const Rotamer& r, const std::vector<V3>& xmoved, const std::vector<V3>& x,
                double bump_dist, double eps, bool* bumped_exact, int64_t* first_bump) {
  bool any_exact = false, any_sure = false, any_near = false;
  int64_t first = -1, idx = 0;
  for (auto& pr : r.pairs) {
    double d = norm(xmoved[pr.first] - x[pr.second]);
    if (bumps(d, bump_dist)) {
      any_exact = true;
      if (first < 0) first = idx;
    }
    if (d < bump_dist - eps) any_sure = true;
    else if (d < bump_dist + eps) any_near = true;
    ++idx;
  }
  *bumped_exact = any_exact;
  *first_bump = first;
  if (any_sure) return 1;
  return any_near ? 2 : 0;
}

struct LigandOut {
  int32_t* orient_score;       // [O]
  int32_t* orient_score_lo;    // [O]
  int32_t* orient_score_hi;    // [O]
  int16_t* orient_pick;        // [O * reps * R]
  int16_t* orient_rigid;       // optional [O] rigid-sweep choice per restart
  int32_t* orient_fragile;     // [O] first fragile step (rep*R + r) or -1
  uint8_t* step_fragile;       // optional [O * reps * R]: 1 where the step's pick is fragile
                               // (step 0 also has bit 2 when the rigid choice is)
  uint8_t* bump;               // optional [O * reps * R * A]: 0 free, 1 bumped, 2 uncertain
  int32_t* cand_score;         // optional [O * reps * R * A] exact candidate score (-1 if bumped)
  double* best_xyz;            // [n*3]
  int32_t* best_orient;        // [1]
  int32_t* best_score;         // [1]
  int32_t* best_robust;        // [1] 1 if o* cannot flip under eps
  int64_t* pair_tests_full;    // [1] eligible pair tests of the full sweep
  int64_t* pair_tests_early;   // [1] pair tests when each candidate stops at its first bump,
                               //     charged in whole 32-pair tiles (at most the pair count)
  int64_t* evals;              // [1]
};

// A ligand with its topology, rotamers and centres derived once.
struct Prepared {
  int n = 0, R = 0;
  Topo topo;
  std::vector<Rotamer> rots;
  std::vector<V3> x0;
  V3 c_lig{0, 0, 0}, c_pocket{0, 0, 0};
};

bool prepare(const float* xyz_in, int n, const int32_t* bonds, int nb, const int32_t* rot_bond, int R,
             const Pocket& P, const Params& prm, Prepared& L, std::string& err) {
  L.n = n;
  L.R = R;
  if (!build_topology(n, bonds, nb, L.topo, err)) return false;
  L.rots.assign(R, Rotamer{});
  for (int r = 0; r < R; ++r)
    if (!build_rotamer(L.topo, bonds, nb, rot_bond[r], prm.min_bond_sep, L.rots[r], err)) return false;
  L.x0.resize(n);
  L.c_lig = V3{0, 0, 0};
  for (int a = 0; a < n; ++a) {
    L.x0[a] = V3{(double)xyz_in[3 * a], (double)xyz_in[3 * a + 1], (double)xyz_in[3 * a + 2]};
    L.c_lig = L.c_lig + L.x0[a];
  }
  L.c_lig = (1.0 / n) * L.c_lig;
  L.c_pocket = pocket_centre(P.origin, P.h, P.nx, P.ny, P.nz);
  return true;
}

// One restart o: generate_starting_pose, then `repetitions` passes of optimize_pose.
// picks[reps*R]; optional bump / cand_score [reps*R*A]; returns the final score, its
// eps-interval, the first fragile step (-1: none) and the final coordinates x.
void search_restart(const Prepared& L, const Pocket& P, const Params& prm, double eps, int o, int16_t* picks,
                    uint8_t* bump, int32_t* cand_score, int* score_out, int* lo_out, int* hi_out,
                    int* fragile_out, std::vector<V3>& x, int16_t* rigid_out = nullptr,
                    int64_t* early_pairs = nullptr, uint8_t* step_fragile = nullptr) {
  int16_t rigid_dummy = 0;
  (void)rigid_dummy;
  const double pi = 3.14159265358979323846;
  const int n = L.n, R = L.R, A = prm.n_angles, reps = prm.repetitions;
  M3 Ro = euler_orientation(o, prm.n_alpha, prm.n_beta, prm.n_gamma);
  x.resize(n);
  for (int a = 0; a < n; ++a) x[a] = L.c_pocket + mul(Ro, L.x0[a] - L.c_lig);
  int fragile_step = -1;
  bool rigid_fragile = false;
  if (rigid_out) *rigid_out = 0;
  if (prm.rigid_span > 0) {  // align_ligand: best rigid rotation about the pocket centre
    const int W = 2 * prm.rigid_span + 1, M = W * W * W;
    std::vector<int> sc(M), lo(M), hi(M);
    for (int m = 0; m < M; ++m) {
      const M3 Rm = rigid_candidate(m, prm.rigid_span, prm.rigid_step);
      int s = 0, l0 = 0, h0 = 0;
      for (int a = 0; a < n; ++a) {
        const V3 y = L.c_pocket + mul(Rm, x[a] - L.c_pocket);
        s += cell_value(P, y);
        int l, h;
        cell_range(P, y, eps, &l, &h);
        l0 += l;
        h0 += h;
      }
      sc[m] = s;
      lo[m] = l0;
      hi[m] = h0;
    }
    int best = 0;
    for (int m = 1; m < M; ++m)
      if (sc[m] > sc[best]) best = m;
    for (int m = 0; m < M; ++m) {  // can an eps move change the choice?
      if (m == best) continue;
      if ((m < best && !(hi[m] < lo[best])) || (m > best && !(hi[m] <= lo[best]))) rigid_fragile = true;
    }
    if (rigid_fragile) fragile_step = 0;
    const M3 Rb = rigid_candidate(best, prm.rigid_span, prm.rigid_step);
    for (int a = 0; a < n; ++a) x[a] = L.c_pocket + mul(Rb, x[a] - L.c_pocket);
    if (rigid_out) *rigid_out = best;
  }
  std::vector<V3> xm(n);
  std::vector<int> score(A), lo(A), hi(A), status(A);
  std::vector<char> bumped(A);
  for (int rep = 0; rep < reps; ++rep)
    for (int r = 0; r < R; ++r) {
      const Rotamer& rot = L.rots[r];
      const int step = rep * R + r;
      V3 u = x[rot.q] - x[rot.p];
      u = (1.0 / norm(u)) * u;
      int static_score = 0;
      for (int a = 0; a < n; ++a)
        if (!rot.moving[a]) static_score += cell_value(P, x[a]);
      for (int k = 0; k < A; ++k) {
        double theta = 2.0 * pi * k / A;
        for (int a = 0; a < n; ++a)
          xm[a] = rot.moving[a] ? x[rot.p] + rodrigues(u, theta, x[a] - x[rot.p]) : x[a];
        bool b_exact;
        int64_t first;
        status[k] = bump_status(rot, xm, x, prm.bump_dist, eps, &b_exact, &first);
        bumped[k] = b_exact;
        if (early_pairs) {  // BumpCheck rejects at the first bumping pair (Sec. 3.2)
          const int64_t P = (int64_t)rot.pairs.size();
          *early_pairs += first < 0 ? P : std::min(P, (first / 32 + 1) * 32);
        }
        int s = static_score, slo = 0, shi = 0;
        for (int a = 0; a < n; ++a)
          if (rot.moving[a]) {
            s += cell_value(P, xm[a]);
            int l, h;
            cell_range(P, xm[a], eps, &l, &h);
            slo += l;
            shi += h;
          }
        score[k] = s;
        lo[k] = slo;  // moving-atom part only: the static part is common to every k
        hi[k] = shi;
        if (bump) bump[(size_t)step * A + k] = (uint8_t)status[k];
        if (cand_score) cand_score[(size_t)step * A + k] = b_exact ? -1 : s;
      }
      int kstar = -1;
      for (int k = 0; k < A; ++k)
        if (!bumped[k] && (kstar < 0 || score[k] > score[kstar])) kstar = k;
      picks[step] = (int16_t)kstar;
      // Can an eps perturbation change the pick?  fragile_step keeps the first such step
      // (0 also marks a fragile rigid choice); step_fragile, when asked for, flags every
      // such step along this trajectory, so that an implementation which made the same
      // picks so far can still be compared after a fragile step.
      if (fragile_step < 0 || step_fragile) {
        bool robust;
        if (kstar < 0) {  // every candidate bumped: robust only if every bump is sure
          robust = true;
          for (int k = 0; k < A; ++k)
            if (status[k] != 1) robust = false;
        } else {
          robust = status[kstar] == 0;
          for (int k = 0; k < A && robust; ++k) {
            if (k == kstar || status[k] == 1) continue;
            if (k < kstar && !(hi[k] < lo[kstar])) robust = false;
            if (k > kstar && !(hi[k] <= lo[kstar])) robust = false;
          }
        }
        if (!robust && fragile_step < 0) fragile_step = step;
        if (step_fragile) step_fragile[step] = robust ? 0 : 1;
      }
      if (kstar >= 0) {  // commit the chosen rotation
        double theta = 2.0 * pi * kstar / A;
        V3 xp = x[rot.p];
        for (int a = 0; a < n; ++a)
          if (rot.moving[a]) x[a] = xp + rodrigues(u, theta, x[a] - xp);
      }
    }
  int s = 0, slo = 0, shi = 0;
  for (int a = 0; a < n; ++a) {
    s += cell_value(P, x[a]);
    int l, h;
    cell_range(P, x[a], eps, &l, &h);
    slo += l;
    shi += h;
  }
  if (step_fragile && rigid_fragile && reps * R > 0) step_fragile[0] |= 2;  // bit 1: fragile rigid choice
  *score_out = s;
  *lo_out = slo;
  *hi_out = shi;
  *fragile_out = fragile_step;
}

int dock_ligand(const float* xyz_in, int n, const int32_t* bonds, int nb, const int32_t* rot_bond,
                int R, const Pocket& P, const Params& prm, double eps, const LigandOut& out,
                std::string& err) {
  Prepared L;
  if (!prepare(xyz_in, n, bonds, nb, rot_bond, R, P, prm, L, err)) return 1;
  const int O = prm.n_alpha * prm.n_beta * prm.n_gamma;
  const int A = prm.n_angles;
  const int reps = prm.repetitions;
  int64_t full_pairs = 0;
  for (auto& r : L.rots) full_pairs += (int64_t)r.pairs.size();
  *out.pair_tests_full = full_pairs * A * reps * O;
  *out.evals = (int64_t)O * reps * R * A;

  std::vector<std::vector<V3>> final_x(O);
  const size_t per_o = (size_t)reps * R;
  int64_t early = 0;
  for (int o = 0; o < O; ++o)
    search_restart(L, P, prm, eps, o, out.orient_pick + o * per_o, out.bump ? out.bump + o * per_o * A : nullptr,
                   out.cand_score ? out.cand_score + o * per_o * A : nullptr, &out.orient_score[o],
                   &out.orient_score_lo[o], &out.orient_score_hi[o], &out.orient_fragile[o], final_x[o],
                   out.orient_rigid ? out.orient_rigid + o : nullptr, &early,
                   out.step_fragile ? out.step_fragile + o * per_o : nullptr);
  *out.pair_tests_early = early;
  int best = 0;
  for (int o = 1; o < O; ++o)
    if (out.orient_score[o] > out.orient_score[best]) best = o;
  bool robust = true;
  for (int o = 0; o < O; ++o) {
    if (out.orient_fragile[o] >= 0) robust = false;
    if (o == best) continue;
    if (o < best && !(out.orient_score_hi[o] < out.orient_score_lo[best])) robust = false;
    if (o > best && !(out.orient_score_hi[o] <= out.orient_score_lo[best])) robust = false;
  }
  *out.best_orient = best;
  *out.best_score = out.orient_score[best];
  *out.best_robust = robust ? 1 : 0;
  for (int a = 0; a < n; ++a) {
    out.best_xyz[3 * a] = final_x[best][a].x;
    out.best_xyz[3 * a + 1] = final_x[best][a].y;
    out.best_xyz[3 * a + 2] = final_x[best][a].z;
  }
  return 0;
}

thread_local std::string g_err;

}  // namespace

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

// ---- single-operation hooks used by the oracle's own pin tests -------------------

void orc_euler(int o, int na, int nb, int ng, double* R9) {
  M3 R = euler_orientation(o, na, nb, ng);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R9[3 * i + j] = R.m[i][j];
}

void orc_rigid_candidate(int m, int span, double step, double* R9) {
  const M3 R = rigid_candidate(m, span, step);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R9[3 * i + j] = R.m[i][j];
}

void orc_rodrigues(const double* u, double theta, const double* v, double* out) {
  V3 r = rodrigues(V3{u[0], u[1], u[2]}, theta, V3{v[0], v[1], v[2]});
  out[0] = r.x;
  out[1] = r.y;
  out[2] = r.z;
}

int orc_score(const uint8_t* grid, int nx, int ny, int nz, double h, const double* origin,
              const double* xyz, int n) {
  Pocket P{grid, nx, ny, nz, h, V3{origin[0], origin[1], origin[2]}};
  int s = 0;
  for (int a = 0; a < n; ++a) s += cell_value(P, V3{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]});
  return s;
}

// Restart pose o: x <- c_pocket + R_o (x - c_lig) (generate_starting_pose).
void orc_place(const float* xyz, int n, int o, int na, int nb, int ng, int nx, int ny, int nz,
               double h, const double* origin, double* out) {
  V3 c_lig{0, 0, 0};
  for (int a = 0; a < n; ++a) c_lig = c_lig + V3{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
  c_lig = (1.0 / n) * c_lig;
  V3 c_pocket = pocket_centre(V3{origin[0], origin[1], origin[2]}, h, nx, ny, nz);
  M3 R = euler_orientation(o, na, nb, ng);
  for (int a = 0; a < n; ++a) {
    V3 y = c_pocket + mul(R, V3{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]} - c_lig);
    out[3 * a] = y.x;
    out[3 * a + 1] = y.y;
    out[3 * a + 2] = y.z;
  }
}

// Fragment of one rotamer: moving[n], *p, *q, and the graph distance matrix dist[n*n].
int orc_fragment(int n, const int32_t* bonds, int nb, int rb, uint8_t* moving, int* p, int* q,
                 int32_t* dist) {
  Topo t;
  Rotamer r;
  if (!build_topology(n, bonds, nb, t, g_err)) return 1;
  if (!build_rotamer(t, bonds, nb, rb, 3, r, g_err)) return 1;
  for (int a = 0; a < n; ++a) moving[a] = (uint8_t)r.moving[a];
  *p = r.p;
  *q = r.q;
  if (dist)
    for (size_t i = 0; i < (size_t)n * n; ++i) dist[i] = t.dist[i];
  return 0;
}

// Apply the rotation of rotamer `rb` by angle index k of A to xyz (in place, FP64).
int orc_torsion(int n, const int32_t* bonds, int nb, int rb, int k, int A, double* xyz) {
  Topo t;
  Rotamer r;
  if (!build_topology(n, bonds, nb, t, g_err)) return 1;
  if (!build_rotamer(t, bonds, nb, rb, 3, r, g_err)) return 1;
  const double pi = 3.14159265358979323846;
  auto X = [&](int a) { return V3{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]}; };
  V3 xp = X(r.p);
  V3 u = X(r.q) - xp;
  u = (1.0 / norm(u)) * u;
  for (int a = 0; a < n; ++a)
    if (r.moving[a]) {
      V3 y = xp + rodrigues(u, 2.0 * pi * k / A, X(a) - xp);
      xyz[3 * a] = y.x;
      xyz[3 * a + 1] = y.y;
      xyz[3 * a + 2] = y.z;
    }
  return 0;
}

// 1 if some moving x static pair of rotamer rb (graph distance >= min_sep) is closer
// than bump_dist in the pose xyz.
int orc_bumped(int n, const int32_t* bonds, int nb, int rb, int min_sep, double bump_dist,
               const double* xyz) {
  Topo t;
  Rotamer r;
  if (!build_topology(n, bonds, nb, t, g_err)) return -1;
  if (!build_rotamer(t, bonds, nb, rb, min_sep, r, g_err)) return -1;
  for (auto& pr : r.pairs) {
    V3 a{xyz[3 * pr.first], xyz[3 * pr.first + 1], xyz[3 * pr.first + 2]};
    V3 b{xyz[3 * pr.second], xyz[3 * pr.second + 1], xyz[3 * pr.second + 2]};
    if (bumps(norm(a - b), bump_dist)) return 1;
  }
  return 0;
}

// ---- features of the learned orientation proposer (FP64) -------------------------
//
// 48 numbers per (ligand, restart o): the restart quaternion (w >= 0), n/250, R/60,
// radius of gyration / 10, 16-bin histogram of centroid distances over [0, 12) A as
// fractions, and grid value / 255 under 25 farthest-point-sampled atoms of the placed
// restart pose.  Farthest-point sampling starts from the atom farthest from the
// centroid; at every step the candidates within a relative 1e-4 of the farthest count
// as tied and the smallest input index wins (the generator's fixed bond geometry makes
// exact ties common).  Also reports how close each decision came to flipping: the
// smallest relative distance of a candidate to that tie threshold, the
// smallest distance of an atom to a histogram bin edge, and a per-sample flag set when
// an eps move of the sampled atom could read another cell value.

static void qmul(const double a[4], const double b[4], double o[4]) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

int orc_features(const float* xyz, int n, int R, int o, int na, int nb, int ng, const uint8_t* grid, int nx, int ny,
                 int nz, double h, const double* origin, double eps, double* feat, int32_t* fps_out, double* fps_gap,
                 double* hist_edge, uint8_t* sample_fragile) {
  const double pi = 3.14159265358979323846;
  if (n < 1) return 1;
  Pocket P{grid, nx, ny, nz, h, V3{origin[0], origin[1], origin[2]}};
  std::vector<V3> x(n);
  V3 c{0, 0, 0};
  for (int a = 0; a < n; ++a) {
    x[a] = V3{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
    c = c + x[a];
  }
  c = (1.0 / n) * c;
  // restart quaternion: qz(alpha) * qy(beta) * qz(gamma), axis-angle halves
  const int i = o / (nb * ng), j = (o / ng) % nb, k = o % ng;
  const double al = 2.0 * pi * i / na, be = pi * (j + 0.5) / nb, ga = 2.0 * pi * k / ng;
  const double qa[4] = {std::cos(al / 2), 0, 0, std::sin(al / 2)};
  const double qb[4] = {std::cos(be / 2), 0, std::sin(be / 2), 0};
  const double qg[4] = {std::cos(ga / 2), 0, 0, std::sin(ga / 2)};
  double t[4], q[4];
  qmul(qa, qb, t);
  qmul(t, qg, q);
  if (q[0] < 0)
    for (double& v : q) v = -v;
  for (int e = 0; e < 4; ++e) feat[e] = q[e];
  feat[4] = n / 250.0;
  feat[5] = R / 60.0;
  double r2 = 0, edge = 1e30;
  for (int e = 0; e < 16; ++e) feat[7 + e] = 0;
  for (int a = 0; a < n; ++a) {
    const double d = norm(x[a] - c);
    r2 += d * d;
    const int b = (int)std::floor(d / 0.75);
    if (b < 16) feat[7 + b] += 1.0 / n;
    edge = std::min(edge, std::fabs(d - 0.75 * std::round(d / 0.75)));
  }
  feat[6] = std::sqrt(r2 / n) / 10.0;
  *hist_edge = edge;
  // farthest-point sampling
  const int nsel = n < 25 ? n : 25;
  std::vector<double> mind(n);
  std::vector<char> used(n, 0);
  std::vector<int> fps;
  double gap = 1e30;
  for (int a = 0; a < n; ++a) mind[a] = norm(x[a] - c);
  for (int s = 0; s < nsel; ++s) {
    // candidates within a relative 1e-4 of the farthest count as tied; smallest index wins
    double dmax = -1;
    for (int a = 0; a < n; ++a)
      if (!used[a]) dmax = std::max(dmax, mind[a]);
    const double thr = (1.0 - 1e-4) * dmax;
    int best = -1;
    for (int a = 0; a < n; ++a) {
      if (used[a]) continue;
      if (best < 0 && mind[a] >= thr) best = a;
      if (dmax > 0) gap = std::min(gap, std::fabs(mind[a] - thr) / dmax);
    }
    used[best] = 1;
    fps.push_back(best);
    for (int a = 0; a < n; ++a) {
      const double d = norm(x[a] - x[best]);
      mind[a] = s == 0 ? d : std::min(mind[a], d);
    }
  }
  *fps_gap = gap;
  const M3 Ro = euler_orientation(o, na, nb, ng);
  const V3 cp = pocket_centre(P.origin, P.h, P.nx, P.ny, P.nz);
  for (int sidx = 0; sidx < 25; ++sidx) {
    const int a = fps[sidx % nsel];
    fps_out[sidx] = a;
    const V3 y = cp + mul(Ro, x[a] - c);
    feat[23 + sidx] = cell_value(P, y) / 255.0;
    int lo, hi;
    cell_range(P, y, eps, &lo, &hi);
    sample_fragile[sidx] = lo != hi;
  }
  return 0;
}

// ---- the whole search over a CSR batch --------------------------------------------

struct orc_params {
  int32_t n_alpha, n_beta, n_gamma, n_angles;
  double bump_dist;
  int32_t min_bond_sep, repetitions;
  int32_t rigid_span;
  double rigid_step;
};

// One restart o of one ligand: picks[reps*R], optional bump/cand_score[reps*R*A],
// score / interval / first fragile step, final coordinates xyz_out[3n], optional
// step_fragile[reps*R] (1 where the step's pick is fragile; bit 2 of step 0: the rigid
// choice is).
int orc_dock_pose(int n, const float* xyz, int nb, const int32_t* bonds, int R, const int32_t* rot_bond,
                  const uint8_t* grid, int nx, int ny, int nz, double h, const double* origin,
                  const orc_params* p, double eps, int o, int16_t* picks, uint8_t* bump, int32_t* cand_score,
                  int32_t* score_lo_hi_fragile, double* xyz_out, uint8_t* step_fragile) {
  Pocket P{grid, nx, ny, nz, h, V3{origin[0], origin[1], origin[2]}};
  Params prm{p->n_alpha, p->n_beta, p->n_gamma, p->n_angles, p->bump_dist, p->min_bond_sep, p->repetitions,
             p->rigid_span, p->rigid_step};
  Prepared L;
  if (!prepare(xyz, n, bonds, nb, rot_bond, R, P, prm, L, g_err)) return 1;
  std::vector<V3> x;
  int16_t rigid = 0;
  search_restart(L, P, prm, eps, o, picks, bump, cand_score, &score_lo_hi_fragile[0], &score_lo_hi_fragile[1],
                 &score_lo_hi_fragile[2], &score_lo_hi_fragile[3], x, &rigid, nullptr, step_fragile);
  score_lo_hi_fragile[4] = rigid;
  for (int a = 0; a < n; ++a) {
    xyz_out[3 * a] = x[a].x;
    xyz_out[3 * a + 1] = x[a].y;
    xyz_out[3 * a + 2] = x[a].z;
  }
  return 0;
}

// Outputs are laid out per ligand i with O = na*nb*ng orientations:
//   orient_* at [i*O ...], picks at [i*O*reps ... ] per rotamer offsets rot_off,
//   best_xyz at [3*atom_off[i] ...]; bump/cand_score (optional) at
//   [(i*O)*reps*Rmax*A ...] is not used -- optional arrays are indexed by
//   cand_off[i] = sum over earlier ligands of O*reps*R*A.
int orc_dock_batch(int L, const int32_t* atom_off, const float* xyz, const int32_t* bond_off,
                   const int32_t* bonds, const int32_t* rot_off, const int32_t* rot_bond,
                   const uint8_t* grid, int nx, int ny, int nz, double h, const double* origin,
                   const orc_params* p, double eps, int n_threads, int32_t* orient_score,
                   int32_t* orient_score_lo, int32_t* orient_score_hi, int16_t* orient_pick,
                   int32_t* orient_fragile, uint8_t* bump, int32_t* cand_score,
                   const int64_t* cand_off, double* best_xyz, int32_t* best_orient,
                   int32_t* best_score, int32_t* best_robust, int64_t* pair_tests_full,
                   int64_t* evals, int32_t* status, int16_t* orient_rigid, int64_t* pair_tests_early,
                   uint8_t* step_fragile) {
  Pocket P{grid, nx, ny, nz, h, V3{origin[0], origin[1], origin[2]}};
  Params prm{p->n_alpha, p->n_beta, p->n_gamma, p->n_angles, p->bump_dist, p->min_bond_sep,
             p->repetitions, p->rigid_span, p->rigid_step};
  const int O = prm.n_alpha * prm.n_beta * prm.n_gamma;
  std::atomic<int> next{0};
  std::vector<std::string> errs(L);
  auto worker = [&]() {
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= L) break;
      LigandOut lo;
      lo.orient_score = orient_score + (size_t)i * O;
      lo.orient_score_lo = orient_score_lo + (size_t)i * O;
      lo.orient_score_hi = orient_score_hi + (size_t)i * O;
      lo.orient_pick = orient_pick + (size_t)rot_off[i] * O * prm.repetitions;
      lo.orient_rigid = orient_rigid ? orient_rigid + (size_t)i * O : nullptr;
      lo.orient_fragile = orient_fragile + (size_t)i * O;
      lo.step_fragile = step_fragile ? step_fragile + (size_t)rot_off[i] * O * prm.repetitions : nullptr;
      lo.bump = bump ? bump + cand_off[i] : nullptr;
      lo.cand_score = cand_score ? cand_score + cand_off[i] : nullptr;
      lo.best_xyz = best_xyz + 3 * (size_t)atom_off[i];
      lo.best_orient = best_orient + i;
      lo.best_score = best_score + i;
      lo.best_robust = best_robust + i;
      lo.pair_tests_full = pair_tests_full + i;
      lo.pair_tests_early = pair_tests_early + i;
      lo.evals = evals + i;
      int n = atom_off[i + 1] - atom_off[i];
      int nb = bond_off[i + 1] - bond_off[i];
      int R = rot_off[i + 1] - rot_off[i];
      status[i] = dock_ligand(xyz + 3 * (size_t)atom_off[i], n, bonds + 2 * (size_t)bond_off[i], nb,
                              rot_bond + rot_off[i], R, P, prm, eps, lo, errs[i]);
    }
  };
  int T = std::max(1, n_threads);
  std::vector<std::thread> pool;
  for (int t = 1; t < T; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < L; ++i)
    if (status[i]) {
      g_err = "ligand " + std::to_string(i) + ": " + errs[i];
      return 1;
    }
  return 0;
}

}  // extern "C"
