// Smoothed-aggregation AMG on the device.
//
// Setup (double precision), for each level l with block size B:
//   1. D = B x B diagonal blocks of S, D^-1, d_i = ||S_ii||_F
//   2. strong directed entries: ||S_ij||_F^2 > theta_l^2 d_i d_j, weight
//      w_ij = ||S_ij||_F^2 / (d_i d_j); the undirected graph is the union of
//      the strong pattern and its transpose with the larger weight
//   3. roots: distance-2 maximal independent set, fixed SplitMix64 keys; a
//      node joins when its key is the largest among undecided nodes within
//      distance 2, which reproduces the greedy set in descending key order
//   4. aggregates: strongest root neighbour, then strongest round-1
//      neighbour, leftovers seed singletons; numbered by seed index
//   5. lambda from 15 normalised power steps of D^-1 S
//   6. P = (I - omega D^-1 S) P_tent with P_tent(i, agg i) = I / sqrt(|agg|)
//   7. R = P^T, S_c = R (S P) by the block SpGEMM (in float in the mixed
//      mode, whose cycle keeps the level operators in float)
// The coarsest operator is inverted explicitly (Gauss-Jordan, partial
// pivoting) in double.
//
// Cycle (float or double): V(1,1), zero initial guess on every level,
// Chebyshev smoother on [cheb_lo * cheb_hi * lambda, cheb_hi * lambda]
// (Saad, Alg. 12.1) fused with the residual in one pass over S.
#include <cmath>
#include <cstdlib>
#include <type_traits>

#include "amg.cuh"

#include <cooperative_groups.h>
namespace cg = cooperative_groups;
#include "sparse.cuh"
#include "spmv.cuh"

namespace fs {

namespace {

constexpr int kT = 256;
inline int grid_rows(int64_t n) { return blocks_for(n, kT, kSMs * 32); }

// levels whose rows hold more blocks than this on average use the
// lane-group BSR kernel instead of sliced ELL (coarse levels)
// blocks of the cooperative Gauss-Jordan launch
#ifndef FS_GJ_MAX_BLOCKS
#define FS_GJ_MAX_BLOCKS 64
#endif
#ifndef FS_SELL_MAX_MEAN_ROW
#define FS_SELL_MAX_MEAN_ROW 40.0
#endif
constexpr double kSellMaxMeanRow = FS_SELL_MAX_MEAN_ROW;
// The forward cycle prolongs through [P | S P], fused with the first
// post-smoothing step; the transposed cycle (adjoint solves) prolongs with P
// alone: as lane-group BSR on levels of at most this many block rows, as
// sliced ELL above
constexpr int kProlongBsrMaxRows = 20000;
// lanes per row of the jagged copies; test hook: FS_JAG_LANES=<g> sets every
// one to g lanes, so that small problems run the lane counts large ones take
inline int jag_lanes_for(int64_t nnzb, int nbr) {
#ifdef FS_TEST_HOOKS
  if (const char *ev = std::getenv("FS_JAG_LANES")) return (int)std::strtol(ev, nullptr, 10);
#endif
  return jag_lanes(nnzb, nbr);
}
// chunked BSR for long-row operators and restrictions; test hook:
// FS_CHUNKED=0 keeps the lane-group BSR kernel, so that a test can compare the two
inline bool chunked_rows() {
#ifdef FS_TEST_HOOKS
  if (const char *ev = std::getenv("FS_CHUNKED")) return std::strtol(ev, nullptr, 10) != 0;
#endif
  return true;
}
// the prolongation fused with the first post-smoothing step; test hook:
// FS_FUSE_PROLONG=0 keeps them apart, so that a test can compare the two
inline bool fuse_prolongation() {
#ifdef FS_TEST_HOOKS
  if (const char *ev = std::getenv("FS_FUSE_PROLONG")) return std::strtol(ev, nullptr, 10) != 0;
#endif
  return true;
}
// scalar hierarchies of at most this many rows run their whole cycle as a graph
constexpr int64_t kWholeGraphMaxRows = 200000;

__device__ inline double frob2(const double *v, int bs) {
  double s = 0.0;
  for (int k = 0; k < bs; k++) s = __dadd_rn(s, __dmul_rn(v[k], v[k]));
  return s;
}

// ------------------------------------------------------------ 1. diagonal
template <int B>
__global__ void k_diag(BsrView<double> S, double *Dinv, double *dn, int *flag) {
  constexpr int BS = B * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int s = S.rp[i], len = S.rp[i + 1] - s;
    int p = find_sorted(S.ci + s, len, (int)i);
    double a[BS];
    for (int k = 0; k < BS; k++) a[k] = p >= 0 ? S.val[(int64_t)(s + p) * BS + k] : 0.0;
    dn[i] = sqrt(frob2(a, BS));
    double *o = Dinv + i * BS;
    if (B == 1) {
      if (!(a[0] != 0.0) || !isfinite(a[0])) { atomicExch(flag, 1); o[0] = 0.0; }
      else o[0] = 1.0 / a[0];
    } else {
      double c00 = a[4] * a[8] - a[5] * a[7];
      double c01 = a[5] * a[6] - a[3] * a[8];
      double c02 = a[3] * a[7] - a[4] * a[6];
      double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
      double sc = 0.0;
      for (int k = 0; k < 9; k++) sc = fmax(sc, fabs(a[k]));
      if (!(fabs(det) > 1e-14 * sc * sc * sc) || !isfinite(det)) {
        atomicExch(flag, 1);
        for (int k = 0; k < 9; k++) o[k] = 0.0;
        continue;
      }
      double id = 1.0 / det;
      o[0] = c00 * id;
      o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
      o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
      o[3] = c01 * id;
      o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
      o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
      o[6] = c02 * id;
      o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
      o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
    }
  }
}

// ------------------------------------------------------------ 2. strength
// pass 0: count strong entries per row; pass 1: write (col, weight)
// Strong couplings of each row, in column order: ||S_ij||_F^2 > theta^2
// ||S_ii||_F ||S_jj||_F (dn holds the diagonal-block norms), weight
// ||S_ij||_F^2 / (||S_ii||_F ||S_jj||_F).  A group of G lanes takes a row and
// G consecutive blocks at a time (coalesced block reads).  Pass 0 evaluates
// every block once, keeps each entry's weight (-1: not strong) in wall and
// counts; pass 1 compacts the strong entries from wall in column order (a
// ballot keeps the order) without reading S's values again.
template <int G>
__global__ void k_strength(BsrView<double> S, const double *dn, double theta2, int pass, int *cnt,
                           double *wall, const int *rpG, int *ciG, double *wG) {
  const int bs = S.br * S.bc;
  const int lane = threadIdx.x & (G - 1);
  const int base = threadIdx.x & 31 & ~(G - 1);
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << base;
  const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G; i < S.nbr; i += ngroups) {
    int n = 0;
    const int o = pass ? rpG[i] : 0;
    const double di = pass ? 0.0 : dn[i];
    const int e1 = S.rp[i + 1];
    for (int eb = S.rp[i]; eb < e1; eb += G) {
      const int e = eb + lane;
      bool strong = false;
      double w = -1.0;
      if (e < e1) {
        if (pass) {
          w = wall[e];
          strong = w >= 0.0;
        } else {
          const int j = S.ci[e];
          if (j != i) {
            const double sv = frob2(S.val + (int64_t)e * bs, bs);
            const double dd = __dmul_rn(di, dn[j]);
            strong = sv > __dmul_rn(theta2, dd);
            if (strong) w = __ddiv_rn(sv, dd);
          }
          wall[e] = w;
        }
      }
      const unsigned m = __ballot_sync(gmask, strong) >> base;
      if (pass && strong) {
        const int pos = n + __popc(m & ((1u << lane) - 1u));
        ciG[o + pos] = S.ci[e];
        wG[o + pos] = w;
      }
      n += __popc(m);
    }
    if (!pass && lane == 0) cnt[i] = n;
  }
}

// union of two sorted weighted patterns, weight = max; pass 0 counts
__global__ void k_union_max(int nr, const int *rpA, const int *ciA, const double *wA, const int *rpB,
                            const int *ciB, const double *wB, int pass, int *cnt, const int *rpC,
                            int *ciC, double *wC) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = rpA[i], ae = rpA[i + 1], b = rpB[i], be = rpB[i + 1];
    int n = 0, o = pass ? rpC[i] : 0;
    while (a < ae || b < be) {
      int ca = a < ae ? ciA[a] : INT32_MAX;
      int cb = b < be ? ciB[b] : INT32_MAX;
      int c = ca < cb ? ca : cb;
      double w = 0.0;
      if (ca == c) { w = fmax(w, wA[a]); a++; }
      if (cb == c) { w = fmax(w, wB[b]); b++; }
      if (pass) { ciC[o + n] = c; wC[o + n] = w; }
      n++;
    }
    if (!pass) cnt[i] = n;
  }
}

// ------------------------------------------------------------ 3. MIS-2
enum : int8_t { ST_UND = 0, ST_ROOT = 1, ST_OUT = 2, ST_NONE = 3 };

__global__ void k_mis_init(int n, const int *rp, uint64_t seed, int level, uint64_t *key, int8_t *st) {
  const uint64_t mask = (1ull << 26) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = sm64_draw(seed, 10, ((uint64_t)level << 32) + (uint64_t)i);
    key[i] = (r & ~mask) | (uint64_t)i;
    st[i] = (rp[i + 1] > rp[i]) ? ST_UND : ST_NONE;
  }
}

// m[v] = 1 + max key over undecided nodes of the closed neighbourhood (0: none)
__global__ void k_mis_max1(int n, const int *rp, const int *ci, const uint64_t *key, const int8_t *st,
                           uint64_t *m) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    uint64_t best = st[v] == ST_UND ? key[v] + 1 : 0;
    for (int e = rp[v]; e < rp[v + 1]; e++) {
      int u = ci[e];
      if (st[u] == ST_UND && key[u] + 1 > best) best = key[u] + 1;
    }
    m[v] = best;
  }
}

__global__ void k_mis_max2_select(int n, const int *rp, const int *ci, const uint64_t *key, const uint64_t *m1,
                                  int8_t *st, int8_t *newroot) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    newroot[v] = 0;
    if (st[v] != ST_UND) continue;
    uint64_t best = m1[v];
    for (int e = rp[v]; e < rp[v + 1]; e++) best = m1[ci[e]] > best ? m1[ci[e]] : best;
    if (best == key[v] + 1) newroot[v] = 1;
  }
}

__global__ void k_mis_mark_near(int n, const int *rp, const int *ci, const int8_t *newroot, int8_t *near) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int8_t x = newroot[v];
    for (int e = rp[v]; e < rp[v + 1] && !x; e++) x = newroot[ci[e]];
    near[v] = x;
  }
}

__global__ void k_mis_update(int n, const int *rp, const int *ci, const int8_t *newroot, const int8_t *near,
                             int8_t *st, int *undecided) {
  int local = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (st[v] != ST_UND) continue;
    if (newroot[v]) { st[v] = ST_ROOT; continue; }
    int8_t x = near[v];
    for (int e = rp[v]; e < rp[v + 1] && !x; e++) x = near[ci[e]];
    if (x) st[v] = ST_OUT;
    else local++;
  }
  if (local) atomicAdd(undecided, local);
}

// ------------------------------------------------------------ 4. aggregates
// round 1: owner = strongest root neighbour (ties: lower index); roots own themselves
__global__ void k_agg_round1(int n, const int *rp, const int *ci, const double *w, const int8_t *st, int *owner) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (st[v] == ST_ROOT) { owner[v] = (int)v; continue; }
    int best = -1;
    double bw = -1.0;
    for (int e = rp[v]; e < rp[v + 1]; e++) {
      int u = ci[e];
      if (st[u] != ST_ROOT) continue;
      if (w[e] > bw || (w[e] == bw && u < best)) { bw = w[e]; best = u; }
    }
    owner[v] = best;
  }
}

// round 2: unassigned nodes join the owner of their strongest assigned neighbour
__global__ void k_agg_round2(int n, const int *rp, const int *ci, const double *w, const int *owner1,
                             int *owner2, int8_t *seed) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int o = owner1[v];
    seed[v] = (o == (int)v) ? 1 : 0;
    if (o >= 0 || rp[v + 1] == rp[v]) { owner2[v] = o; continue; }
    int best = -1;
    double bw = -1.0;
    for (int e = rp[v]; e < rp[v + 1]; e++) {
      int u = ci[e];
      if (owner1[u] < 0) continue;
      if (w[e] > bw || (w[e] == bw && u < best)) { bw = w[e]; best = u; }
    }
    if (best >= 0) owner2[v] = owner1[best];
    else { owner2[v] = (int)v; seed[v] = 1; }   // leftover seeds a singleton
  }
}

__global__ void k_seed_flags_to_int(int n, const int8_t *seed, int *out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    out[v] = seed[v];
}

__global__ void k_agg_number(int n, const int *owner, const int *seedidx, int *agg, int *size) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int o = owner[v];
    int a = o >= 0 ? seedidx[o] : -1;
    agg[v] = a;
    if (a >= 0) atomicAdd(size + a, 1);
  }
}

// ------------------------------------------------------------ 5. power
__global__ void k_power_start(int64_t n, uint64_t seed, int level, double *v) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    v[k] = 2.0 * sm64_uniform(seed, 11, ((uint64_t)level << 32) + (uint64_t)k) - 1.0;
}

// ------------------------------------------------------------ 6. prolongator
// 1 / sqrt|a| of every aggregate (the scale of its tentative block), once
__global__ void k_inv_sqrt_size(const int *asize, int nc, double *isz) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nc; a += (int64_t)gridDim.x * blockDim.x)
    isz[a] = 1.0 / sqrt((double)asize[a]);
}

// One warp per row i of S.  The aggregates a(j) of the row's columns are
// staged in shared memory; the distinct ones, ranked in increasing order, are
// the row's columns in P.  For each distinct a, the blocks S_ij with
// a(j) = a are added in row order, then
//   P_ia = [a(i) = a] I / sqrt|a| - omega D_i^-1 (sum_j S_ij) / sqrt|a|.
template <int B>
__global__ void k_prolong(BsrView<double> S, const int *agg, const double *isz_agg, const double *Dinv,
                          double omega, int pass, int *cnt, const int *rpP, int *ciP, double *valP,
                          int cap, int *flag) {
  constexpr int BS = B * B;
  extern __shared__ int sh_agg[];
  __shared__ double sh_sum[8][32 * BS];        // short rows: block sums per aggregate (at most 8 warps)
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  int *al = sh_agg + (size_t)wid * 3 * cap;   // aggregate of entry t (-1: none)
  int *fl = al + cap;                          // 1 if entry t is the first with its aggregate
  int *rk = fl + cap;                          // rank of that aggregate among the distinct ones
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  for (int64_t i = blockIdx.x * (int64_t)wpb + wid; i < S.nbr; i += nwarps) {
    const int s0 = S.rp[i], len = S.rp[i + 1] - s0;
    if (len > cap) {
      if (lane == 0) { atomicExch(flag, 1); if (!pass) cnt[i] = 0; }
      continue;
    }
    if (len <= 32) {
      // short rows: one entry per lane; lanes with equal aggregates found
      // by a match, ranks by counting the distinct smaller aggregates
      const int a = lane < len ? agg[S.ci[s0 + lane]] : -1;
      const unsigned act = __ballot_sync(0xffffffffu, lane < len);
      const unsigned same = __match_any_sync(0xffffffffu, a);
      const bool first = lane < len && a >= 0 && (same & ((1u << lane) - 1u)) == 0;
      const unsigned firsts = __ballot_sync(0xffffffffu, first);
      int r = 0;
      for (unsigned m = firsts; m; m &= m - 1) {
        const int u = __ffs(m) - 1;
        r += __shfl_sync(0xffffffffu, a, u) < a;
      }
      const int nu = __popc(firsts);
      (void)act;
      if (!pass) {
        if (lane == 0) cnt[i] = nu;
        continue;
      }
      // the B x B entries of the row's nu blocks of P, spread over the lanes
      // (unit k: aggregate number k / BS in lane order, entry k % BS).  First
      // each entry of an aggregate's block sum, in row order, as a whole
      // block would; then D_i^-1 times the scaled sums
      const int o = rpP[i];
      const double *Di = Dinv + i * BS;
      const int ai = agg[i];
      const double isz_first = first ? isz_agg[a] : 0.0;
      double *sums = sh_sum[wid];
      for (int k0 = 0; k0 < nu * BS; k0 += 32) {
        const int k = k0 + lane;
        const int fi = min(k / BS, nu - 1), e = k - (k / BS) * BS;
        unsigned m = firsts;   // lane holding the fi-th first entry
        for (int t = 0; t < fi; t++) m &= m - 1;
        const unsigned fsame = __shfl_sync(0xffffffffu, same, __ffs(m) - 1);
        if (k < nu * BS) {
          double acc = 0.0;
          for (unsigned mu = fsame; mu; mu &= mu - 1) acc += S.val[(int64_t)(s0 + __ffs(mu) - 1) * BS + e];
          sums[k] = acc;
        }
      }
      __syncwarp();
      for (int k0 = 0; k0 < nu * BS; k0 += 32) {
        const int k = k0 + lane;
        const int fi = min(k / BS, nu - 1), e = k - (k / BS) * BS;
        unsigned m = firsts;
        for (int t = 0; t < fi; t++) m &= m - 1;
        const int fl = __ffs(m) - 1;
        const int fa = __shfl_sync(0xffffffffu, a, fl);
        const int fr = __shfl_sync(0xffffffffu, r, fl);
        const double isz = __shfl_sync(0xffffffffu, isz_first, fl);
        if (k < nu * BS) {
          const int rr = e / B, cc = e - rr * B;
          double mm = 0.0;
#pragma unroll
          for (int q = 0; q < B; q++) mm += Di[rr * B + q] * (sums[fi * BS + q * B + cc] * isz);
          const double pt = (ai == fa && rr == cc) ? isz : 0.0;
          valP[(int64_t)(o + fr) * BS + e] = pt - omega * mm;
          if (e == 0) ciP[o + fr] = fa;
        }
      }
      __syncwarp();
      continue;
    }
    for (int t = lane; t < len; t += 32) al[t] = agg[S.ci[s0 + t]];
    __syncwarp();
    for (int t = lane; t < len; t += 32) {
      const int a = al[t];
      bool first = a >= 0;
      for (int u = 0; u < t && first; u++) first = (al[u] != a);
      fl[t] = first;
    }
    __syncwarp();
    int nu = 0;
    for (int t = lane; t < len; t += 32) {
      int r = -1;
      if (fl[t]) {
        const int a = al[t];
        r = 0;
        for (int u = 0; u < len; u++) r += (fl[u] && al[u] < a);
        nu++;
      }
      rk[t] = r;
    }
    for (int o = 16; o > 0; o >>= 1) nu += __shfl_xor_sync(0xffffffffu, nu, o);
    __syncwarp();
    if (!pass) {
      if (lane == 0) cnt[i] = nu;
      __syncwarp();
      continue;
    }
    const int o = rpP[i];
    const double *Di = Dinv + i * BS;
    const int ai = agg[i];
    for (int t = lane; t < len; t += 32) {
      const int r = rk[t];
      if (r < 0) continue;
      const int a = al[t];
      double acc[BS];
      for (int q = 0; q < BS; q++) acc[q] = 0.0;
      for (int u = t; u < len; u++) {
        if (al[u] != a) continue;
        const double *v = S.val + (int64_t)(s0 + u) * BS;
        for (int q = 0; q < BS; q++) acc[q] += v[q];
      }
      const double isz = isz_agg[a];
      double *out = valP + (int64_t)(o + r) * BS;
      for (int rr = 0; rr < B; rr++)
        for (int cc = 0; cc < B; cc++) {
          double m = 0.0;
          for (int q = 0; q < B; q++) m += Di[rr * B + q] * (acc[q * B + cc] * isz);
          const double pt = (ai == a && rr == cc) ? isz : 0.0;
          out[rr * B + cc] = pt - omega * m;
        }
      ciP[o + r] = a;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ 7. coarsest
__global__ void k_bsr_to_dense(BsrView<double> S, double *Dn) {
  const int B = S.br, n = S.nbr * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S.nbr;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int e = S.rp[i]; e < S.rp[i + 1]; e++) {
      int j = S.ci[e];
      for (int r = 0; r < B; r++)
        for (int c = 0; c < B; c++)
          Dn[(i * B + r) * (int64_t)n + j * B + c] = S.val[(int64_t)e * B * B + r * B + c];
    }
}

// Gauss-Jordan step k, part 1 (one block): partial pivoting (lowest index on
// ties), row swap, scaling of the pivot row, copy of column k
// One Gauss-Jordan pivot step on a single block of 1024 threads (shared
// arrays sv, si of blockDim entries): choose the pivot row, swap it into
// row k, scale row k and save the multipliers of column k.
__device__ void gj_pivot_step(double *M, int n, int k, int *perm, double *colk, int *flag, double *sv,
                              int *si) {
  double best = -1.0;
  int bi = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(M[(int64_t)i * n + k]);
    if (v > best || (v == best && i < bi)) { best = v; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v = sv[threadIdx.x + o];
      int ii = si[threadIdx.x + o];
      if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && ii < si[threadIdx.x])) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = ii;
      }
    }
    __syncthreads();
  }
  const int p = si[0];
  if (threadIdx.x == 0) {
    perm[k] = p;
    if (!(sv[0] > 0.0)) atomicExch(flag, 1);
  }
  if (p != k && p < n)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = M[(int64_t)k * n + j];
      M[(int64_t)k * n + j] = M[(int64_t)p * n + j];
      M[(int64_t)p * n + j] = t;
    }
  __syncthreads();
  double piv = M[(int64_t)k * n + k];
  double ip = piv != 0.0 ? 1.0 / piv : 0.0;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double v = (j == k) ? ip : M[(int64_t)k * n + j] * ip;
    M[(int64_t)k * n + j] = v;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = (i == k) ? 0.0 : M[(int64_t)i * n + k];
}

__global__ void k_gj_pivot(double *M, int n, int k, int *perm, double *colk, int *flag) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  gj_pivot_step(M, n, k, perm, colk, flag, sv, si);
}

// part 2: a_ij -= a_ik a_kj for i != k (column k becomes -a_ik / piv)
__device__ inline void gj_elim_step(double *M, int n, int k, const double *colk) {
  int64_t total = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / n), j = (int)(t - (int64_t)i * n);
    if (i == k) continue;
    double f = colk[i];
    double base = (j == k) ? 0.0 : M[t];
    M[t] = base - f * M[(int64_t)k * n + j];
  }
}

__global__ void k_gj_elim(double *M, int n, int k, const double *colk) { gj_elim_step(M, n, k, colk); }

// All n steps in one cooperative launch (co-resident blocks, one grid-wide
// barrier per step): step k reads matrix Mk and writes Mn (ping-pong), so
// every block can take the pivot of column k itself (the same search, the
// same row) and eliminate its entries without waiting for a pivot phase.
// The arithmetic per entry is that of the two-kernel step: the pivot row
// (swapped into row k) scaled by 1/piv, then a_ij - a_ik a~_kj with column k
// becoming -a_ik / piv.  perm[k] = pivot row; the result ends in buf[n & 1].
__global__ void __launch_bounds__(1024) k_gj_coop(double *buf0, double *buf1, int n, int *perm, int *flag) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  cg::grid_group grid = cg::this_grid();
  for (int k = 0; k < n; k++) {
    const double *Mk = (k & 1) ? buf1 : buf0;
    double *Mn = (k & 1) ? buf0 : buf1;
    double best = -1.0;
    int bi = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      double v = fabs(Mk[(int64_t)i * n + k]);
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        double v = sv[threadIdx.x + o];
        int ii = si[threadIdx.x + o];
        if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && ii < si[threadIdx.x])) {
          sv[threadIdx.x] = v;
          si[threadIdx.x] = ii;
        }
      }
      __syncthreads();
    }
    const int p = si[0] < n ? si[0] : k;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      perm[k] = p;
      if (!(sv[0] > 0.0)) atomicExch(flag, 1);
    }
    const double piv = Mk[(int64_t)p * n + k];
    const double ip = piv != 0.0 ? 1.0 / piv : 0.0;
    __syncthreads();
    const int64_t total = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
      const int i = (int)(t / n), j = (int)(t - (int64_t)i * n);
      const double rkj = (j == k) ? ip : Mk[(int64_t)p * n + j] * ip;   // scaled pivot row
      if (i == k) {
        Mn[t] = rkj;
      } else {
        const int src = (i == p) ? k : i;                                  // rows k and p swap
        const double aik = Mk[(int64_t)src * n + k];
        const double base = (j == k) ? 0.0 : Mk[(int64_t)src * n + j];
        Mn[t] = base - aik * rkj;
      }
    }
    grid.sync();
  }
}

__global__ void k_gj_unpermute(double *M, int n, const int *perm) {
  // undo the row interchanges by swapping columns in reverse order
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double *row = M + (int64_t)i * n;
    for (int k = n - 1; k >= 0; k--) {
      int p = perm[k];
      if (p != k) {
        double t = row[k];
        row[k] = row[p];
        row[p] = t;
      }
    }
  }
}

// ------------------------------------------------------------ cycle kernels
template <int B, typename TP>
__global__ void k_cheb_zero(int64_t nb, const TP *f, const TP *Dinv, TP cr, TP *d, TP *x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    TP fi[B];
#pragma unroll
    for (int q = 0; q < B; q++) fi[q] = f[i * B + q];
    const TP *D = Dinv + i * B * B;
#pragma unroll
    for (int a = 0; a < B; a++) {
      TP s = 0;
#pragma unroll
      for (int b = 0; b < B; b++) s += D[a * B + b] * fi[b];
      TP v = cr * s;
      d[i * B + a] = v;
      x[i * B + a] = v;
    }
  }
}

// x = Cinv f in double, one warp per row
template <typename TP>
__global__ void k_dense_gemv(int n, const double *__restrict__ M, const TP *__restrict__ f, TP *x) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += M[i * n + j] * (double)f[j];
    s = warp_sum(s);
    if (lane == 0) x[i] = (TP)s;
  }
}

}  // namespace

// ============================================================ setup driver
namespace {

struct Graph {
  DBuf<int> rp, ci;
  DBuf<double> w;
  int n = 0;
  int64_t nnz = 0;
};

Graph strength_graph(const BsrView<double> &S, const double *dn, double theta, cudaStream_t s) {
  const int n = S.nbr;
  Graph Gd;
  Gd.n = n;
  Gd.rp.alloc(n + 1);
  DBuf<int> cnt(n + 1);
  const double th2 = theta * theta;
  constexpr int SG = 8;   // lanes per row
  const int sgrid = blocks_for((int64_t)n * SG, kT, kSMs * 32);
  DBuf<double> wall(S.nnzb > 0 ? S.nnzb : 1);
  k_strength<SG><<<sgrid, kT, 0, s>>>(S, dn, th2, 0, cnt.p, wall.p, nullptr, nullptr, nullptr);
  FS_LAUNCHED();
  Gd.nnz = exclusive_scan(cnt.p, Gd.rp.p, n, s);
  Gd.ci.alloc(Gd.nnz);
  Gd.w.alloc(Gd.nnz);
  if (Gd.nnz) {
    k_strength<SG><<<sgrid, kT, 0, s>>>(S, dn, th2, 1, nullptr, wall.p, Gd.rp.p, Gd.ci.p, Gd.w.p);
    FS_LAUNCHED();
  }
  // transpose of the directed strong pattern (weights as 1x1 blocks)
  BsrView<double> gv;
  gv.nbr = n; gv.nbc = n; gv.br = 1; gv.bc = 1; gv.nnzb = Gd.nnz;
  gv.rp = Gd.rp.p; gv.ci = Gd.ci.p; gv.val = Gd.w.p;
  Bsr<double> Gt = transpose(gv, s);
  Graph G;
  G.n = n;
  G.rp.alloc(n + 1);
  k_union_max<<<grid_rows(n), kT, 0, s>>>(n, Gd.rp.p, Gd.ci.p, Gd.w.p, Gt.rp.p, Gt.ci.p, Gt.val.p, 0,
                                          cnt.p, nullptr, nullptr, nullptr);
  FS_LAUNCHED();
  G.nnz = exclusive_scan(cnt.p, G.rp.p, n, s);
  G.ci.alloc(G.nnz);
  G.w.alloc(G.nnz);
  if (G.nnz) {
    k_union_max<<<grid_rows(n), kT, 0, s>>>(n, Gd.rp.p, Gd.ci.p, Gd.w.p, Gt.rp.p, Gt.ci.p, Gt.val.p,
                                            1, nullptr, G.rp.p, G.ci.p, G.w.p);
    FS_LAUNCHED();
  }
  return G;
}

// returns the number of aggregates; agg filled (-1 = none), asize filled
int aggregate(const Graph &G, uint64_t seed, int level, DBuf<int> &agg, DBuf<int> &asize, int verbose,
              cudaStream_t s) {
  const int n = G.n;
  FS_REQUIRE(n < (1 << 26) - 1, FC_BAD_ARG, "AMG level too large for 26-bit node keys");
  DBuf<uint64_t> key(n), m1(n);
  DBuf<int8_t> st(n), newroot(n), nearf(n);
  DBuf<int> und(1);
  k_mis_init<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, seed, level, key.p, st.p);
  FS_LAUNCHED();
  int rounds = 0;
  for (;;) {
    FS_CUDA(cudaMemsetAsync(und.p, 0, sizeof(int), s));
    k_mis_max1<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, G.ci.p, key.p, st.p, m1.p);
    FS_LAUNCHED();
    k_mis_max2_select<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, G.ci.p, key.p, m1.p, st.p, newroot.p);
    FS_LAUNCHED();
    k_mis_mark_near<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, G.ci.p, newroot.p, nearf.p);
    FS_LAUNCHED();
    k_mis_update<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, G.ci.p, newroot.p, nearf.p, st.p, und.p);
    FS_LAUNCHED();
    int h = 0;
    FS_CUDA(cudaMemcpyAsync(&h, und.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    rounds++;
    if (h == 0) break;
    FS_REQUIRE(rounds < 10000, FC_INTERNAL, "MIS-2 did not terminate");
  }
  DBuf<int> owner1(n), owner2(n), seedi(n), seedidx(n + 1);
  DBuf<int8_t> seedf(n);
  k_agg_round1<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, G.ci.p, G.w.p, st.p, owner1.p);
  FS_LAUNCHED();
  k_agg_round2<<<grid_rows(n), kT, 0, s>>>(n, G.rp.p, G.ci.p, G.w.p, owner1.p, owner2.p, seedf.p);
  FS_LAUNCHED();
  k_seed_flags_to_int<<<grid_rows(n), kT, 0, s>>>(n, seedf.p, seedi.p);
  FS_LAUNCHED();
  int nc = (int)exclusive_scan(seedi.p, seedidx.p, n, s);
  agg.alloc(n);
  asize.alloc(nc > 0 ? nc : 1);
  FS_CUDA(cudaMemsetAsync(asize.p, 0, sizeof(int) * (nc > 0 ? nc : 1), s));
  k_agg_number<<<grid_rows(n), kT, 0, s>>>(n, owner2.p, seedidx.p, agg.p, asize.p);
  FS_LAUNCHED();
  if (verbose) fprintf(stderr, "[fracsolve] level %d: %d nodes, %d aggregates, %d MIS rounds\n", level, n, nc, rounds);
  return nc;
}

template <typename TP>
__global__ void k_power_scale(TP *v, const TP *w, int64_t n, const double *ww, const double *vv, double *lam) {
  const double nw = sqrt(*ww);
  const double a = 1.0 / nw;
  if (blockIdx.x == 0 && threadIdx.x == 0) *lam = nw / sqrt(*vv);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    v[k] = (TP)(a * (double)w[k]);
}

template <int B, typename TP, typename Epi>
void op_apply(const SellView<TP> &S, const TP *v, const Epi &e, cudaStream_t s) {
  sell_spmv<B, B>(S, v, e, s);
}
template <int B, typename TP, typename Epi>
void op_apply(const BsrView<TP> &S, const TP *v, const Epi &e, cudaStream_t s) {
  spmv<B, B>(S, v, e, s);
}

// lambda of D^-1 S by normalised power steps on the cycle-precision operator
// (in the layout the cycle uses for it); norms in double on the device, one
// host read at the end
template <int B, typename TP, typename M>
double power_lambda(const M &S, const TP *Dinv, uint64_t seed, int level, int steps, cudaStream_t s) {
  const int64_t n = (int64_t)S.nbr * B;
  DBuf<double> v0(n), scal(2 + steps), part(kRedBlocks + 1);
  DBuf<TP> v(n), w(n);
  k_power_start<<<grid_rows(n), kT, 0, s>>>(n, seed, level, v0.p);
  FS_LAUNCHED();
  cast(v.p, v0.p, n, s);
  for (int it = 0; it < steps; it++) {
    EpiBlockDiag<B, TP> e{w.p, Dinv};
    op_apply<B, TP>(S, v.p, e, s);
    nrm2sq_dev(w.p, n, scal.p, s, part.p);
    nrm2sq_dev(v.p, n, scal.p + 1, s, part.p);
    k_power_scale<TP><<<grid_rows(n), kT, 0, s>>>(v.p, w.p, n, scal.p, scal.p + 1, scal.p + 2 + it);
    FS_LAUNCHED();
  }
  double lam = 0.0;
  FS_CUDA(cudaMemcpyAsync(&lam, scal.p + 1 + steps, sizeof(double), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(std::isfinite(lam) && lam > 0, FC_NAN, "power iteration broke down");
  return lam;
}

__global__ void k_max_len_rows(const int *rp, int n, int *out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, rp[i + 1] - rp[i]);
  atomicMax(out, m);
}

template <int B>
void build_prolongator(LevelSetup &L, const DBuf<int> &asize, int nc, double omega, cudaStream_t s) {
  const BsrView<double> S = L.S.view();
  Bsr<double> &P = L.P;
  P.shape(L.nb, nc, B, B);
  P.rp.alloc(L.nb + 1);
  DBuf<int> cnt(L.nb + 1), flag(2);
  FS_CUDA(cudaMemsetAsync(flag.p, 0, 2 * sizeof(int), s));
  k_max_len_rows<<<blocks_for(L.nb, 256, kSMs * 4), 256, 0, s>>>(S.rp, L.nb, flag.p + 1);
  FS_LAUNCHED();
  int hl[2] = {0, 0};
  FS_CUDA(cudaMemcpyAsync(hl, flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  const int cap = hl[1] > 0 ? hl[1] : 1;
  FS_REQUIRE(cap <= 4096, FC_INTERNAL, "level operator row longer than 4096 blocks");
  int wpb = 8;
  while (wpb > 1 && (size_t)wpb * 3 * cap * sizeof(int) > 96 * 1024) wpb >>= 1;
  const size_t shm = (size_t)wpb * 3 * cap * sizeof(int);
  FS_CUDA(cudaFuncSetAttribute(k_prolong<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const int grid = kSMs * 8;
  DBuf<double> isz(nc > 0 ? nc : 1);
  if (nc > 0) {
    k_inv_sqrt_size<<<blocks_for(nc, 256, kSMs * 4), 256, 0, s>>>(asize.p, nc, isz.p);
    FS_LAUNCHED();
  }
  k_prolong<B><<<grid, wpb * 32, shm, s>>>(S, L.agg.p, isz.p, L.Dinv.p, omega, 0, cnt.p, nullptr, nullptr,
                                            nullptr, cap, flag.p);
  FS_LAUNCHED();
  P.nnzb = exclusive_scan(cnt.p, P.rp.p, L.nb, s);
  P.ci.alloc(P.nnzb);
  P.val.alloc(P.nnzb * B * B);
  if (P.nnzb) {
    k_prolong<B><<<grid, wpb * 32, shm, s>>>(S, L.agg.p, isz.p, L.Dinv.p, omega, 1, nullptr, P.rp.p, P.ci.p,
                                              P.val.p, cap, flag.p);
    FS_LAUNCHED();
  }
  FS_CUDA(cudaMemcpyAsync(hl, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!hl[0], FC_INTERNAL, "prolongator row exceeds the shared capacity");
}

// Values of the smoothed prolongator on its existing pattern (the pattern
// depends only on the pattern of S and the aggregates).
template <int B>
void prolongator_values(LevelSetup &L, double omega, cudaStream_t s) {
  const BsrView<double> S = L.S.view();
  Bsr<double> &P = L.P;
  DBuf<int> flag(2);
  FS_CUDA(cudaMemsetAsync(flag.p, 0, 2 * sizeof(int), s));
  k_max_len_rows<<<blocks_for(L.nb, 256, kSMs * 4), 256, 0, s>>>(S.rp, L.nb, flag.p + 1);
  FS_LAUNCHED();
  int hl[2] = {0, 0};
  FS_CUDA(cudaMemcpyAsync(hl, flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  const int cap = hl[1] > 0 ? hl[1] : 1;
  FS_REQUIRE(cap <= 4096, FC_INTERNAL, "level operator row longer than 4096 blocks");
  int wpb = 8;
  while (wpb > 1 && (size_t)wpb * 3 * cap * sizeof(int) > 96 * 1024) wpb >>= 1;
  const size_t shm = (size_t)wpb * 3 * cap * sizeof(int);
  FS_CUDA(cudaFuncSetAttribute(k_prolong<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  DBuf<double> isz(L.nc > 0 ? L.nc : 1);
  if (L.nc > 0) {
    k_inv_sqrt_size<<<blocks_for(L.nc, 256, kSMs * 4), 256, 0, s>>>(L.asize.p, L.nc, isz.p);
    FS_LAUNCHED();
  }
  if (P.nnzb) {
    k_prolong<B><<<kSMs * 8, wpb * 32, shm, s>>>(S, L.agg.p, isz.p, L.Dinv.p, omega, 1, nullptr, P.rp.p,
                                                 P.ci.p, P.val.p, cap, flag.p);
    FS_LAUNCHED();
  }
  FS_CUDA(cudaMemcpyAsync(hl, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!hl[0], FC_INTERNAL, "prolongator row exceeds the shared capacity");
}

void invert_coarsest(Hierarchy &H, cudaStream_t s) {
  LevelSetup &L = H.lev.back();
  const int n = L.nb * L.B;
  H.nc_scalar = n;
  H.cinv.alloc((size_t)n * n > 0 ? (size_t)n * n : 1);
  if (n == 0) return;
  FS_CUDA(cudaMemsetAsync(H.cinv.p, 0, sizeof(double) * (size_t)n * n, s));
  k_bsr_to_dense<<<grid_rows(L.nb), kT, 0, s>>>(L.S.view(), H.cinv.p);
  FS_LAUNCHED();
  DBuf<int> perm(n), flag(1);
  DBuf<double> colk(n);
  FS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  int dev = 0, coop = 0, per_sm = 0;
  FS_CUDA(cudaGetDevice(&dev));
  FS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (coop) FS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_coop, 1024, 0));
  if (coop && per_sm > 0) {
    int nsm = 0;
    FS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // few blocks: the grid-wide barrier per step costs more with every block
    const int want = (int)std::min<int64_t>(std::min<int64_t>(((int64_t)n * n + 1023) / 1024, (int64_t)nsm * per_sm),
                                            FS_GJ_MAX_BLOCKS);
    const int blocks = std::max(1, want);
    DBuf<double> other((size_t)n * n);
    double *b0 = H.cinv.p, *b1 = other.p;
    int *pp = perm.p, *fp = flag.p;
    int nn = n;
    void *args[] = {&b0, &b1, &nn, &pp, &fp};
    FS_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_coop, dim3(blocks), dim3(1024), args, 0, s));
    FS_LAUNCHED();
    if (n & 1)
      FS_CUDA(cudaMemcpyAsync(H.cinv.p, other.p, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    FS_CUDA(cudaStreamSynchronize(s));
  } else {
    const int eg = blocks_for((int64_t)n * n, 256, kSMs * 8);
    for (int k = 0; k < n; k++) {
      k_gj_pivot<<<1, 1024, 0, s>>>(H.cinv.p, n, k, perm.p, colk.p, flag.p);
      FS_LAUNCHED();
      k_gj_elim<<<eg, 256, 0, s>>>(H.cinv.p, n, k, colk.p);
      FS_LAUNCHED();
    }
  }
  k_gj_unpermute<<<blocks_for(n, 128, kSMs), 128, 0, s>>>(H.cinv.p, n, perm.p);
  FS_LAUNCHED();
  int h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!h, FC_SINGULAR_BLOCK, "singular coarsest-level matrix");
}

template <typename TP>
void prepare_cycle(Hierarchy &H, std::vector<LevelCycle<TP>> &C, cudaStream_t s) {
  C.clear();
  C.resize(H.lev.size());
  for (size_t l = 0; l < H.lev.size(); l++) {
    LevelSetup &L = H.lev[l];
    LevelCycle<TP> &c = C[l];
    const int64_t n = (int64_t)L.nb * L.B;
    const bool last = (l + 1 == H.lev.size());
    const bool sell = L.nb == 0 || (double)L.S.nnzb / L.nb <= kSellMaxMeanRow;
    if constexpr (std::is_same<TP, double>::value) {
      c.S = L.S.view();
      if (!last) { c.P = L.P.view(); c.R = L.R.view(); c.Dinv = L.Dinv.p; }
      if (sell) c.Ss = L.Ssd.nbr == L.nb && L.Ssd.sp.p ? std::move(L.Ssd) : to_sell<TP>(L.S.view(), s);
    } else {
      if (!last) {
        c.R_own = copy_cast<TP, double>(L.R.view(), s);
        c.R = c.R_own.view();
        if (L.Dinvf.p) {
          c.Dinv_own = std::move(L.Dinvf);
        } else {
          c.Dinv_own.alloc((size_t)L.nb * L.B * L.B);
          cast(c.Dinv_own.p, L.Dinv.p, (int64_t)L.nb * L.B * L.B, s);
        }
        c.Dinv = c.Dinv_own.p;
      }
      if (sell) {
        c.Ss = L.Ssf.nbr == L.nb && L.Ssf.sp.p ? std::move(L.Ssf) : to_sell<TP>(L.S.view(), s);
      } else {
        if constexpr (std::is_same<TP, float>::value) {
          if (L.Sbf.nbr == L.nb && L.Sbf.val.p) c.S_own = std::move(L.Sbf);
          else c.S_own = copy_cast<TP, double>(L.S.view(), s);
        } else {
          c.S_own = copy_cast<TP, double>(L.S.view(), s);
        }
        c.S = c.S_own.view();
      }
    }
    L.Ssf = Sell<float>();
    L.Ssd = Sell<double>();
    L.Sbf = Bsr<float>();
    c.op.sell = sell;
    c.op.sv = c.Ss.view();
    c.op.bv = c.S;
    c.op.nnzb = L.S.nnzb;
    c.op.nbr = L.nb;
    if (!sell && !last && chunked_rows() && !rowcta_rows(L.S.nnzb, L.nb)) {
      c.Sk = to_chunked<TP>(L.S.view(), lanes_for(L.S.nnzb, L.nb, L.B * L.B), s);
      c.op.chunk = true;
      c.op.kv = c.Sk.view();
    }
    if (!last) {
      c.Ps = to_sell<TP>(L.P.view(), s);
      // levels with few rows prolong through the lane-group BSR kernel: a
      // warp per 32-row slice leaves most of the GPU idle there
      if (L.nb <= kProlongBsrMaxRows) {
        if constexpr (std::is_same<TP, double>::value) c.P = L.P.view();
        else {
          c.P_own = copy_cast<TP, double>(L.P.view(), s);
          c.P = c.P_own.view();
        }
      } else {
        c.P = BsrView<TP>();
      }
      if (chunked_rows() && L.R.nbr > 0 && !rowcta_rows(L.R.nnzb, L.R.nbr))
        c.Rk = to_chunked<TP>(L.R.view(), lanes_for(L.R.nnzb, L.R.nbr, L.B * L.B), s);
      // the prolongation and the first post-smoothing step read P and S P
      // (in the cycle precision: S P is formed in it by the Galerkin product)
      if (fuse_prolongation() && L.nb > 0) {
        if constexpr (std::is_same<TP, float>::value) {
          if (L.SPf.nbr == L.nb && L.SPf.rp.p) {
            const BsrView<float> q = L.SPf.view();
            c.PSP = to_jag<float, float>(L.P.view(), &q, jag_lanes_for(L.P.nnzb + q.nnzb, L.nb), s);
          }
        } else {
          if (L.SP.nbr == L.nb && L.SP.rp.p) {
            const BsrView<double> q = L.SP.view();
            c.PSP = to_jag<double, double>(L.P.view(), &q, jag_lanes_for(L.P.nnzb + q.nnzb, L.nb), s);
          }
        }
      }
    }
    c.f.alloc(n > 0 ? n : 1);
    c.x.alloc(n > 0 ? n : 1);
    c.xa.alloc(n > 0 ? n : 1);
    c.d.alloc(n > 0 ? n : 1);
    c.r.alloc(n > 0 ? n : 1);
    if (!last) {
      double hi = H.prm.cheb_hi * L.lam, lo = H.prm.cheb_lo * hi;
      c.theta = 0.5 * (hi + lo);
      c.delta = 0.5 * (hi - lo);
      c.sigma = c.theta / c.delta;
    }
  }
  FS_CUDA(cudaStreamSynchronize(s));
}

// D^-1 of level l (3x3 or 1x1 block inverses); dn receives the block norms
// the strength test uses.
template <int B>
void level_diag(LevelSetup &L, int l, DBuf<double> &dn, cudaStream_t s) {
  const int nb = L.nb;
  L.Dinv.alloc((size_t)nb * B * B);
  dn.alloc(nb > 0 ? nb : 1);
  DBuf<int> flag(1);
  FS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  k_diag<B><<<grid_rows(nb), kT, 0, s>>>(L.S.view(), L.Dinv.p, dn.p, flag.p);
  FS_LAUNCHED();
  int hf = 0;
  FS_CUDA(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!hf, FC_SINGULAR_BLOCK, "singular diagonal block in AMG level " + std::to_string(l));
}

// power estimate of the largest eigenvalue of D^-1 S on the sliced-ELL copy
// of S in the cycle precision (the copy is handed to the cycle afterwards)
template <int B>
void level_lambda(LevelSetup &L, const AmgParams &p, int l, int precision, cudaStream_t s) {
  const int nb = L.nb;
  const bool sell = nb == 0 || (double)L.S.nnzb / nb <= kSellMaxMeanRow;
  if (precision == FC_MIXED) {
    L.Dinvf.alloc((size_t)nb * B * B);
    cast(L.Dinvf.p, L.Dinv.p, (int64_t)nb * B * B, s);
    if (sell) {
      L.Ssf = to_sell<float>(L.S.view(), s);
      L.lam = power_lambda<B, float>(L.Ssf.view(), L.Dinvf.p, p.seed, l, p.power_steps, s);
    } else {
      L.Sbf = copy_cast<float, double>(L.S.view(), s);
      L.lam = power_lambda<B, float>(L.Sbf.view(), L.Dinvf.p, p.seed, l, p.power_steps, s);
    }
  } else if (sell) {
    L.Ssd = to_sell<double>(L.S.view(), s);
    L.lam = power_lambda<B, double>(L.Ssd.view(), L.Dinv.p, p.seed, l, p.power_steps, s);
  } else {
    L.lam = power_lambda<B, double>(L.S.view(), L.Dinv.p, p.seed, l, p.power_steps, s);
  }
}

// The Galerkin product S_c = R (S P).  In the mixed mode, whose cycle
// stores and applies every level operator in float, the block products and
// their sums run in float: the double SpGEMM is bound by this part's FP64
// FMA rate (1/64 of FP32).  The float result is widened to double for the
// next level's setup (strength, aggregation, prolongator).  The FP64 mode
// keeps the double products.  numeric_only: the patterns of S P and S_c are
// those of an earlier call (a numeric rebuild).
void galerkin(LevelSetup &L, Bsr<double> &Sc, int precision, bool numeric_only, cudaStream_t s) {
  if (precision != FC_MIXED) {
    if (numeric_only) {
      spgemm_numeric(L.S.view(), L.P.view(), L.SP, s);
      spgemm_numeric(L.R.view(), L.SP.view(), Sc, s);
    } else {
      L.SP = spgemm(L.S.view(), L.P.view(), s);
      Sc = spgemm(L.R.view(), L.SP.view(), s);
    }
    return;
  }
  const Bsr<float> Sf = copy_cast<float, double>(L.S.view(), s);
  const Bsr<float> Pf = copy_cast<float, double>(L.P.view(), s);
  const Bsr<float> Rf = copy_cast<float, double>(L.R.view(), s);
  if (numeric_only) {
    spgemm_numeric(Sf.view(), Pf.view(), L.SPf, s);
    Bsr<float> Scf = copy_cast<float, double>(Sc.view(), s);   // the pattern of S_c
    spgemm_numeric(Rf.view(), L.SPf.view(), Scf, s);
    cast(Sc.val.p, Scf.val.p, Sc.nnzb * Sc.br * Sc.bc, s);
  } else {
    L.SPf = spgemm(Sf.view(), Pf.view(), s);
    const Bsr<float> Scf = spgemm(Rf.view(), L.SPf.view(), s);
    Sc = copy_cast<double, float>(Scf.view(), s);
  }
  FS_CUDA(cudaStreamSynchronize(s));   // the float temporaries go out of scope here
}

template <int B>
void setup_levels(Hierarchy &H, Bsr<double> &&S0, int precision, cudaStream_t s) {
  const AmgParams &p = H.prm;
  H.lev.clear();
  H.lev.emplace_back();
  H.lev[0].B = B;
  H.lev[0].S = std::move(S0);
  H.lev[0].nb = H.lev[0].S.nbr;
  PhaseTimer pt(p.verbose > 0, s, B == 3 ? "amg3" : "amg1");
  for (int l = 0;; l++) {
    LevelSetup &L = H.lev[l];
    const int nb = L.nb;
    if (p.verbose) fprintf(stderr, "[fracsolve] AMG(B=%d) level %d: %d block rows, %lld blocks\n", B, l, nb, (long long)L.S.nnzb);
    if (nb <= p.coarse_max || l + 1 >= p.max_levels) break;
    DBuf<double> dn;
    level_diag<B>(L, l, dn, s);
    pt.mark("diag");
    // strength graph and aggregates
    const double theta = p.theta0 * std::pow(p.theta_decay, l);
    Graph G = strength_graph(L.S.view(), dn.p, theta, s);
    pt.mark("strength");
    int nc = aggregate(G, p.seed, l, L.agg, L.asize, p.verbose, s);
    pt.mark("aggregate");
    if (nc == 0 || nc > p.max_ratio * nb) {
      L.Dinv.release();
      L.agg.release();
      L.asize.release();
      break;
    }
    L.nc = nc;
    level_lambda<B>(L, p, l, precision, s);
    pt.mark("power");
    build_prolongator<B>(L, L.asize, nc, p.omega_num / L.lam, s);
    pt.mark("prolongator");
    L.R = transpose(L.P.view(), s);
    pt.mark("transpose");
    Bsr<double> Sc;
    galerkin(L, Sc, precision, false, s);
    pt.mark("Galerkin R (S P)");
    LevelSetup next;
    next.B = B;
    next.S = std::move(Sc);
    next.nb = nc;
    H.lev.push_back(std::move(next));
  }
  const int nlast = H.lev.back().nb * B;
  FS_REQUIRE(nlast <= 8192, FC_INTERNAL, "coarsest AMG level too large for the dense solve");
  invert_coarsest(H, s);
  pt.mark("coarsest inverse");
  if (precision == FC_MIXED) prepare_cycle<float>(H, H.cf, s);
  else prepare_cycle<double>(H, H.cd, s);
  pt.mark("cycle data");
  H.built = true;
}

// Numeric rebuild on new values of the level-0 operator with the same
// pattern: aggregates, tentative prolongators and every sparsity pattern of
// the hierarchy are kept; D^-1, lambda, the smoothed prolongator values, R,
// the Galerkin products (numeric pass only), the coarsest inverse and the
// cycle data are recomputed.
template <int B>
void refresh_levels(Hierarchy &H, Bsr<double> &&S0, int precision, cudaStream_t s) {
  const AmgParams &p = H.prm;
  H.built = false;
  H.lev[0].S = std::move(S0);
  PhaseTimer pt(p.verbose > 0, s, B == 3 ? "amg3 refresh" : "amg1 refresh");
  const int nl = (int)H.lev.size();
  for (int l = 0; l + 1 < nl; l++) {
    LevelSetup &L = H.lev[l];
    DBuf<double> dn;
    level_diag<B>(L, l, dn, s);
    level_lambda<B>(L, p, l, precision, s);
    pt.mark("diag + power");
    prolongator_values<B>(L, p.omega_num / L.lam, s);
    L.R = transpose(L.P.view(), s);
    pt.mark("prolongator + transpose");
    galerkin(L, H.lev[l + 1].S, precision, true, s);
    pt.mark("spgemm numeric");
  }
  invert_coarsest(H, s);
  if (precision == FC_MIXED) prepare_cycle<float>(H, H.cf, s);
  else prepare_cycle<double>(H, H.cd, s);
  pt.mark("coarsest + cycle data");
  H.built = true;
}

}  // namespace

void amg_refresh(Hierarchy &H, Bsr<double> &&S0, int precision, cudaStream_t s) {
  NvtxRange nvtx("amg_refresh");
  FS_REQUIRE(H.built && !H.lev.empty(), FC_NOT_SETUP, "AMG hierarchy not built");
  const Bsr<double> &S = H.lev[0].S;
  FS_REQUIRE(S0.nbr == S.nbr && S0.nnzb == S.nnzb && S0.br == S.br, FC_BAD_ARG,
             "AMG refresh: the operator's pattern differs from the one the hierarchy was built on");
  FS_REQUIRE(same_pattern(S0.view(), S.view(), s), FC_BAD_ARG,
             "AMG refresh: the operator's pattern differs from the one the hierarchy was built on");
  for (auto &row : H.coarse)
    for (auto &g : row) g.reset();
  for (auto &g : H.whole) g.reset();
  H.have_t = false;
  if (H.B == 3) refresh_levels<3>(H, std::move(S0), precision, s);
  else refresh_levels<1>(H, std::move(S0), precision, s);
}

void amg_setup(Hierarchy &H, Bsr<double> &&S0, int B, const AmgParams &prm, int precision,
               cudaStream_t s) {
  NvtxRange nvtx("amg_setup");
  H.prm = prm;
  H.B = B;
  H.built = false;
  H.graphs = prm.graphs;
  for (auto &row : H.coarse)
    for (auto &g : row) g.reset();
  for (auto &g : H.whole) g.reset();
  if (B == 3) setup_levels<3>(H, std::move(S0), precision, s);
  else if (B == 1) setup_levels<1>(H, std::move(S0), precision, s);
  else throw Error(FC_BAD_ARG, "AMG block size must be 1 or 3");
}

// ============================================================ cycle
namespace {
// algorithmic bytes of one fused Chebyshev step: the operator (values,
// column indices, row pointers), the iterate gathered once, f, d read and
// written, the new iterate and the inverse diagonal blocks
template <int B, typename TP>
double cheb_bytes(const LevelOp<TP> &S, bool read_d) {
  const double sz = sizeof(TP);
  return (double)S.nnzb * (B * B * sz + 4) + (double)(S.nbr + 1) * 4 +
         (double)S.nbr * B * sz * (read_d ? 5 : 4) + (double)S.nbr * B * B * sz;
}

template <int BR, int BC, typename TP, typename TX, typename Epi>
inline void op_spmv(const LevelOp<TP> &A, const TX *x, const Epi &e, cudaStream_t s) {
  if (A.chunk) chunk_spmv<BR, BC>(A.kv, x, e, s);
  else if (A.sell) sell_spmv<BR, BC>(A.sv, x, e, s);
  else spmv<BR, BC>(A.bv, x, e, s);
}
template <int BR, int BC, typename TP, typename TX, typename TY, typename TZ>
inline void op_axpby(const LevelOp<TP> &A, const TX *x, TY *y, double alpha, double beta, const TZ *z,
                     cudaStream_t s) {
  EpiAxpby<BR, TP, TY, TZ> e{y, z, (TP)alpha, (TP)beta};
  op_spmv<BR, BC>(A, x, e, s);
}


template <int B, typename TP, bool TR = false>
void cycle_level(Hierarchy &H, std::vector<LevelCycle<TP>> &C, int l, const TP *f, TP *xout, cudaStream_t s);

// Levels 1 .. of the cycle (level-1 f in, level-1 x out) replayed as one CUDA
// graph: the coarse levels are many short kernels whose launch cost exceeds
// their run time.  Captured on a private stream at the first use.
template <int B, typename TP, bool TR>
void coarse_graph(Hierarchy &H, std::vector<LevelCycle<TP>> &C, cudaStream_t s) {
  GraphExec &ge = H.coarse[sizeof(TP) == 8 ? 1 : 0][TR ? 1 : 0];
  if (!ge.g) {
    cudaStream_t cs = nullptr;
    FS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const unsigned long long k0 = launch_count();
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        cycle_level<B, TP, TR>(H, C, 1, C[1].f.p, C[1].x.p, cs);
      } catch (...) {
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        throw;
      }
      e = cudaStreamEndCapture(cs, &g);
    }
    const unsigned long long captured = launch_count() - k0;
    add_launches(-(long long)captured);   // recorded, not run
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.g, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    FS_CUDA(e);
    ge.kernels = captured;
  }
  FS_CUDA(cudaGraphLaunch(ge.g, s));
  add_launches((long long)ge.kernels);
}

template <int B, typename TP, bool TR>
void cycle_level(Hierarchy &H, std::vector<LevelCycle<TP>> &C, int l, const TP *f, TP *xout, cudaStream_t s) {
  const int L = (int)C.size();
  if (l == L - 1) {
    const int n = H.nc_scalar;
    if (n == 0) return;
    k_dense_gemv<TP><<<blocks_for((int64_t)n * 32, 256, kSMs * 16), 256, 0, s>>>(n, TR ? H.cinvT.p : H.cinv.p,
                                                                                 f, xout);
    FS_LAUNCHED();
    return;
  }
  LevelCycle<TP> &c = C[l];
  const LevelOp<TP> &Sop = TR ? c.opT : c.op;
  const TP *Dv = TR ? c.DinvT.p : c.Dinv;
  const int64_t nb = c.op.nbr;
  const int deg = H.prm.cheb_degree;
  TP *buf[2] = {c.xa.p, xout};
  int cur = 0;
  // pre-smoothing from x = 0
  double rho = 1.0 / c.sigma;
  k_cheb_zero<B, TP><<<grid_rows(nb), kT, 0, s>>>(nb, f, Dv, (TP)(1.0 / c.theta), c.d.p, buf[cur]);
  FS_LAUNCHED();
  Profiler *pf = (l == 0 && !TR) ? H.prof : nullptr;
  for (int k = 1; k < deg; k++) {
    double rn = 1.0 / (2.0 * c.sigma - rho);
    EpiCheb<B, TP> e{f, buf[cur], buf[1 - cur], c.d.p, Dv, (TP)(rn * rho), (TP)(2.0 * rn / c.delta)};
    if (pf) pf->start(PK_SMOOTH0, s);
    op_spmv<B, B>(Sop, buf[cur], e, s);
    if (pf) pf->stop(PK_SMOOTH0, s, cheb_bytes<B, TP>(c.op, true));
    cur ^= 1;
    rho = rn;
  }
  // residual, restriction, coarse correction, prolongation
  if (pf) pf->start(PK_RESID0, s);
  op_axpby<B, B>(Sop, buf[cur], c.r.p, -1.0, 1.0, f, s);
  if (pf) pf->stop(PK_RESID0, s, cheb_bytes<B, TP>(c.op, false) - (double)c.op.nbr * B * B * sizeof(TP));
  LevelCycle<TP> &cn = C[l + 1];
  if (pf) pf->start(PK_RESTRICT0, s);
  if (c.Rk.nbr > 0) {
    EpiAxpby<B, TP, TP, TP> e{cn.f.p, nullptr, (TP)1, (TP)0};
    chunk_spmv<B, B>(c.Rk.view(), c.r.p, e, s);
  } else {
    spmv_axpby<B, B>(c.R, c.r.p, cn.f.p, 1.0, 0.0, (const TP *)nullptr, s);
  }
  if (pf) pf->stop(PK_RESTRICT0, s, (double)c.R.nnzb * (B * B * sizeof(TP) + 4) + (double)c.R.nbr * 4);
  if (pf) pf->start(PK_COARSE0, s);
  if (l == 0 && H.graphs && L > 2) coarse_graph<B, TP, TR>(H, C, s);
  else cycle_level<B, TP, TR>(H, C, l + 1, cn.f.p, cn.x.p, s);
  if (pf) pf->stop(PK_COARSE0, s, 0.0);
  rho = 1.0 / c.sigma;
  if (!TR && c.PSP.nbr > 0) {
    // prolongation and the first post-smoothing step in one pass: the
    // residual of the corrected iterate is r - (S P) x_c
    EpiProlongCheb<B, TP> e{buf[cur], c.r.p, Dv, buf[1 - cur], c.d.p, (TP)(1.0 / c.theta)};
    if (pf) pf->start(PK_PROLONG0, s);
    jag2_spmv<B, B>(c.PSP.view(), cn.x.p, e, s);
    if (pf)
      pf->stop(PK_PROLONG0, s,
               (double)c.PSP.nnzb * (B * B * sizeof(TP) + 4) + (double)c.PSP.nbr * (8 + 5 * B * sizeof(TP)) +
                   (double)c.PSP.nbr * B * B * sizeof(TP));
    cur ^= 1;
  } else {
    if (pf) pf->start(PK_PROLONG0, s);
    if (c.P.nbr > 0) spmv_axpby<B, B>(c.P, cn.x.p, buf[cur], 1.0, 1.0, buf[cur], s);
    else sell_axpby<B, B>(c.Ps.view(), cn.x.p, buf[cur], 1.0, 1.0, buf[cur], s);
    if (pf) pf->stop(PK_PROLONG0, s, (double)c.Ps.nnzb * (B * B * sizeof(TP) + 4) + (double)c.Ps.nbr * 4);
    // post-smoothing from the corrected iterate
    EpiCheb<B, TP> e{f, buf[cur], buf[1 - cur], c.d.p, Dv, (TP)0, (TP)(1.0 / c.theta)};
    if (pf) pf->start(PK_SMOOTH0, s);
    op_spmv<B, B>(Sop, buf[cur], e, s);
    if (pf) pf->stop(PK_SMOOTH0, s, cheb_bytes<B, TP>(c.op, false));
    cur ^= 1;
  }
  for (int k = 1; k < deg; k++) {
    double rn = 1.0 / (2.0 * c.sigma - rho);
    EpiCheb<B, TP> e{f, buf[cur], buf[1 - cur], c.d.p, Dv, (TP)(rn * rho), (TP)(2.0 * rn / c.delta)};
    if (pf) pf->start(PK_SMOOTH0, s);
    op_spmv<B, B>(Sop, buf[cur], e, s);
    if (pf) pf->stop(PK_SMOOTH0, s, cheb_bytes<B, TP>(c.op, true));
    cur ^= 1;
    rho = rn;
  }
}
}  // namespace

template <typename TP>
void amg_vcycle(Hierarchy &H, const TP *f, TP *x, cudaStream_t s) {
  NvtxRange nvtx("vcycle");
  FS_REQUIRE(H.built, FC_NOT_SETUP, "AMG hierarchy not built");
  std::vector<LevelCycle<TP>> *C;
  if constexpr (std::is_same<TP, float>::value) C = &H.cf;
  else C = &H.cd;
  FS_REQUIRE(!C->empty(), FC_NOT_SETUP, "AMG cycle data not prepared for this precision");
  if (H.B == 3) {
    cycle_level<3, TP>(H, *C, 0, f, x, s);
    return;
  }
  // a small scalar hierarchy (T or S~2: a few ten thousand rows) is all
  // short kernels: its whole cycle replays as one graph on the level-0
  // buffers, f copied in and x copied out
  LevelCycle<TP> &c0 = (*C)[0];
  const int64_t n0 = (int64_t)H.lev[0].nb;
  if (!H.graphs || C->size() < 2 || n0 > kWholeGraphMaxRows || n0 == 0) {
    cycle_level<1, TP>(H, *C, 0, f, x, s);
    return;
  }
  GraphExec &ge = H.whole[sizeof(TP) == 8 ? 1 : 0];
  if (!ge.g) {
    cudaStream_t cs = nullptr;
    FS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const unsigned long long k0 = launch_count();
    H.graphs = false;   // no nested capture of the coarse levels
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        cycle_level<1, TP>(H, *C, 0, c0.f.p, c0.x.p, cs);
      } catch (...) {
        H.graphs = true;
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        throw;
      }
      e = cudaStreamEndCapture(cs, &g);
    }
    H.graphs = true;
    const unsigned long long captured = launch_count() - k0;
    add_launches(-(long long)captured);   // recorded, not run
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.g, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    FS_CUDA(e);
    ge.kernels = captured;
  }
  FS_CUDA(cudaMemcpyAsync(c0.f.p, f, sizeof(TP) * n0, cudaMemcpyDeviceToDevice, s));
  FS_CUDA(cudaGraphLaunch(ge.g, s));
  add_launches((long long)ge.kernels);
  FS_CUDA(cudaMemcpyAsync(x, c0.x.p, sizeof(TP) * n0, cudaMemcpyDeviceToDevice, s));
}

template void amg_vcycle<float>(Hierarchy &, const float *, float *, cudaStream_t);
template void amg_vcycle<double>(Hierarchy &, const double *, double *, cudaStream_t);

namespace {
template <typename T>
__global__ void k_transpose_blocks(int64_t nb, int B, const T *in, T *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < B; r++)
      for (int c = 0; c < B; c++) out[i * B * B + c * B + r] = in[i * B * B + r * B + c];
}
__global__ void k_transpose_dense(int n, const double *in, double *out) {
  int64_t total = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / n), j = (int)(t - (int64_t)i * n);
    out[(int64_t)j * n + i] = in[t];
  }
}

template <typename TP>
void prepare_transpose(Hierarchy &H, std::vector<LevelCycle<TP>> &C, cudaStream_t s) {
  for (size_t l = 0; l < H.lev.size(); l++) {
    LevelSetup &L = H.lev[l];
    LevelCycle<TP> &c = C[l];
    if (l + 1 == H.lev.size()) break;   // the coarsest level uses cinvT
    Bsr<double> St = transpose(L.S.view(), s);
    c.opT.sell = c.op.sell;
    c.opT.nnzb = c.op.nnzb;
    c.opT.nbr = c.op.nbr;
    if (c.op.sell) {
      c.SsT = to_sell<TP>(St.view(), s);
      c.opT.sv = c.SsT.view();
    } else {
      c.St_own = copy_cast<TP, double>(St.view(), s);
      c.opT.bv = c.St_own.view();
    }
    const int64_t nb = L.nb;
    c.DinvT.alloc((size_t)nb * L.B * L.B);
    k_transpose_blocks<TP><<<blocks_for(nb, 256, kSMs * 8), 256, 0, s>>>(nb, L.B, c.Dinv, c.DinvT.p);
    FS_LAUNCHED();
  }
  const int n = H.nc_scalar;
  H.cinvT.alloc((size_t)n * n > 0 ? (size_t)n * n : 1);
  if (n) {
    k_transpose_dense<<<blocks_for((int64_t)n * n, 256, kSMs * 8), 256, 0, s>>>(n, H.cinv.p, H.cinvT.p);
    FS_LAUNCHED();
  }
  FS_CUDA(cudaStreamSynchronize(s));
}
}  // namespace

void amg_prepare_transpose(Hierarchy &H, int precision, cudaStream_t s) {
  FS_REQUIRE(H.built, FC_NOT_SETUP, "AMG hierarchy not built");
  if (H.have_t) return;
  if (precision == FC_MIXED) prepare_transpose<float>(H, H.cf, s);
  else prepare_transpose<double>(H, H.cd, s);
  H.have_t = true;
}

template <typename TP>
void amg_vcycle_t(Hierarchy &H, const TP *f, TP *x, cudaStream_t s) {
  NvtxRange nvtx("vcycle_t");
  FS_REQUIRE(H.built && H.have_t, FC_NOT_SETUP, "transposed AMG cycle not prepared");
  std::vector<LevelCycle<TP>> *C;
  if constexpr (std::is_same<TP, float>::value) C = &H.cf;
  else C = &H.cd;
  FS_REQUIRE(!C->empty(), FC_NOT_SETUP, "AMG cycle data not prepared for this precision");
  if (H.B == 3) cycle_level<3, TP, true>(H, *C, 0, f, x, s);
  else cycle_level<1, TP, true>(H, *C, 0, f, x, s);
}
template void amg_vcycle_t<float>(Hierarchy &, const float *, float *, cudaStream_t);
template void amg_vcycle_t<double>(Hierarchy &, const double *, double *, cudaStream_t);

}  // namespace fs
