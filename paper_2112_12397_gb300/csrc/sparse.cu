// Setup-phase sparse kernels: transpose, block SpGEMM, sparse add.
#include "sparse.cuh"
#include "sell.cuh"

namespace fs {

// ============================================================ transpose
namespace {
__global__ void k_count_cols(const int *ci, int64_t nnz, int *cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + ci[e], 1);
}

// scatter entries (row i, col j) to row j of the transpose; order inside a
// transposed row is fixed afterwards by k_sort_rows
__global__ void k_scatter_t(BsrView<double> A, const int *rpT, int *cursor, int *ciT, int64_t *src) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int e = A.rp[i]; e < A.rp[i + 1]; e++) {
      int j = A.ci[e];
      int pos = rpT[j] + atomicAdd(cursor + j, 1);
      ciT[pos] = (int)i;
      src[pos] = e;
    }
  }
}

// Sort each row by column, carrying the source index: one warp per row ranks
// its entries in shared memory (rank = number of smaller columns; columns in
// a transposed row are distinct); rows above the shared capacity fall back
// to an insertion sort by one lane.
__global__ void k_sort_rows(int nr, const int *rp, int *ci, int64_t *src, int cap) {
  extern __shared__ int64_t sh_src[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  int64_t *ws = sh_src + (size_t)wid * cap;
  int *wc = reinterpret_cast<int *>(sh_src + (size_t)wpb * cap) + (size_t)wid * cap;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  for (int64_t i = blockIdx.x * (int64_t)wpb + wid; i < nr; i += nwarps) {
    const int s = rp[i], e = rp[i + 1], len = e - s;
    if (len <= 1) continue;
    if (len <= cap) {
      for (int t = lane; t < len; t += 32) { wc[t] = ci[s + t]; ws[t] = src[s + t]; }
      __syncwarp();
      for (int t = lane; t < len; t += 32) {
        const int key = wc[t];
        int rank = 0;
        for (int u = 0; u < len; u++) rank += (wc[u] < key);
        ci[s + rank] = key;
        src[s + rank] = ws[t];
      }
      __syncwarp();
    } else if (lane == 0) {
      for (int a = s + 1; a < e; a++) {
        int key = ci[a];
        int64_t ks = src[a];
        int b = a - 1;
        while (b >= s && ci[b] > key) {
          ci[b + 1] = ci[b];
          src[b + 1] = src[b];
          b--;
        }
        ci[b + 1] = key;
        src[b + 1] = ks;
      }
    }
    __syncwarp();
  }
}

__global__ void k_max_len(const int *rp, int n, int *out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, rp[i + 1] - rp[i]);
  atomicMax(out, m);
}

__global__ void k_gather_t(int64_t nnz, const int64_t *src, const double *val, int br, int bc,
                           double *valT) {
  int bs = br * bc;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double *v = val + src[p] * bs;
    double *o = valT + p * bs;
    // block (br x bc) -> (bc x br)
    for (int r = 0; r < br; r++)
      for (int c = 0; c < bc; c++) o[c * br + r] = v[r * bc + c];
  }
}
}  // namespace

Bsr<double> transpose(const BsrView<double> &A, cudaStream_t s) {
  Bsr<double> T;
  T.shape(A.nbc, A.nbr, A.bc, A.br);
  T.rp.alloc(A.nbc + 1);
  DBuf<int> cnt(A.nbc + 1);
  FS_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (A.nbc + 1), s));
  if (A.nnzb > 0) {
    k_count_cols<<<blocks_for(A.nnzb, 256, kSMs * 8), 256, 0, s>>>(A.ci, A.nnzb, cnt.p);
    FS_LAUNCHED();
  }
  int64_t nnz = exclusive_scan(cnt.p, T.rp.p, A.nbc, s);
  T.nnzb = nnz;
  T.ci.alloc(nnz);
  T.val.alloc(nnz * A.br * A.bc);
  if (nnz == 0) return T;
  DBuf<int64_t> src(nnz);
  FS_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (A.nbc + 1), s));
  k_scatter_t<<<blocks_for(A.nbr, 128, kSMs * 8), 128, 0, s>>>(A, T.rp.p, cnt.p, T.ci.p, src.p);
  FS_LAUNCHED();
  {
    DBuf<int> mx(1);
    FS_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(int), s));
    k_max_len<<<blocks_for(A.nbc, 256, kSMs * 4), 256, 0, s>>>(T.rp.p, A.nbc, mx.p);
    FS_LAUNCHED();
    int umax = 0;
    FS_CUDA(cudaMemcpyAsync(&umax, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    const size_t per = sizeof(int64_t) + sizeof(int);
    int cap = umax > 1 ? umax : 2, wpb = 8;
    while (wpb > 1 && (size_t)wpb * cap * per > 192 * 1024) wpb >>= 1;
    if ((size_t)wpb * cap * per > 192 * 1024) cap = (int)(192 * 1024 / per);
    const size_t shm = (size_t)wpb * cap * per;
    FS_CUDA(cudaFuncSetAttribute(k_sort_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_sort_rows<<<kSMs * 4, wpb * 32, shm, s>>>(A.nbc, T.rp.p, T.ci.p, src.p, cap);
    FS_LAUNCHED();
  }
  k_gather_t<<<blocks_for(nnz, 256, kSMs * 8), 256, 0, s>>>(nnz, src.p, A.val, A.br, A.bc, T.val.p);
  FS_LAUNCHED();
  FS_CUDA(cudaStreamSynchronize(s));
  return T;
}

// ============================================================ SpGEMM
namespace {
constexpr int kHashCap = 1024;     // per-warp hash slots (power of two)
constexpr int kListCap = 768;      // unique columns a row may hold
constexpr int kWarpsPerBlock = 4;

struct WarpHash {
  int *keys;   // kHashCap
  int *list;   // kListCap
  int *count;  // 1
};

__device__ inline void hash_clear(WarpHash &h, int lane) {
  for (int k = lane; k < kHashCap; k += 32) h.keys[k] = -1;
  if (lane == 0) *h.count = 0;
  __syncwarp();
}

// returns false on overflow
__device__ inline bool hash_insert(WarpHash &h, int key) {
  unsigned slot = ((unsigned)key * 2654435761u) & (kHashCap - 1);
  for (int probe = 0; probe < kHashCap; probe++) {
    int old = atomicCAS(h.keys + slot, -1, key);
    if (old == -1) {
      int pos = atomicAdd(h.count, 1);
      if (pos >= kListCap) return false;
      h.list[pos] = key;
      return true;
    }
    if (old == key) return true;
    slot = (slot + 1) & (kHashCap - 1);
  }
  return false;
}

// Prefix of the B-row lengths over the row of A (a0, na): pre[x] = products
// of entries 0..x-1, pre[na] = T (returned to every lane).
__device__ inline int row_product_prefix(const BsrView<double> &A, const BsrView<double> &B, int a0, int na,
                                         int *pre, int lane) {
  int run = 0;
  for (int x0 = 0; x0 < na; x0 += 32) {
    const int x = x0 + lane;
    int len = 0;
    if (x < na) {
      const int k = A.ci[a0 + x];
      len = B.rp[k + 1] - B.rp[k];
    }
    int inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (x < na) pre[x + 1] = run + inc;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) pre[0] = 0;
  __syncwarp();
  return run;
}

// Product t of the row (enumeration order: entries of A's row, then the
// entries of the matching B row): the A entry offset x with pre[x] <= t < pre[x+1].
__device__ inline int product_entry(const int *pre, int na, int t) {
  int lo = 0, hi = na - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kSymPre = 512;   // A-row entries the flattened symbolic pass takes

// pass 0: count unique columns per row; pass 1: write sorted columns.  The
// products of a row are enumerated flat (all lanes busy even when the rows
// of B are short); rows of A longer than kSymPre take the entry-by-entry loop.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_spgemm_symbolic(BsrView<double> A, BsrView<double> B, int pass, int *cnt, const int *rpC,
                      int *ciC, int *overflow) {
  __shared__ int s_keys[kWarpsPerBlock][kHashCap];
  __shared__ int s_list[kWarpsPerBlock][kListCap];
  __shared__ int s_pre[kWarpsPerBlock][kSymPre + 1];
  __shared__ int s_cnt[kWarpsPerBlock];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpHash h{s_keys[wid], s_list[wid], &s_cnt[wid]};
  int *pre = s_pre[wid];
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t i = blockIdx.x * (int64_t)kWarpsPerBlock + wid; i < A.nbr; i += nwarps) {
    hash_clear(h, lane);
    bool ok = true;
    const int a0 = A.rp[i], na = A.rp[i + 1] - a0;
    if (na <= kSymPre) {
      const int T = row_product_prefix(A, B, a0, na, pre, lane);
      for (int t = lane; t < T; t += 32) {
        const int x = product_entry(pre, na, t);
        const int k = A.ci[a0 + x];
        ok &= hash_insert(h, B.ci[B.rp[k] + (t - pre[x])]);
      }
    } else {
      for (int e = a0; e < a0 + na; e++) {
        int k = A.ci[e];
        for (int f = B.rp[k] + lane; f < B.rp[k + 1]; f += 32) ok &= hash_insert(h, B.ci[f]);
      }
    }
    __syncwarp();
    ok = __all_sync(0xffffffffu, ok);
    int u = *h.count;
    if (!ok || u > kListCap) {
      if (lane == 0) atomicExch(overflow, 1);
      __syncwarp();
      continue;
    }
    if (pass == 0) {
      if (lane == 0) cnt[i] = u;
    } else {
      int base = rpC[i];
      for (int a = lane; a < u; a += 32) {
        int key = h.list[a];
        int rank = 0;
        for (int b = 0; b < u; b++) rank += (h.list[b] < key);
        ciC[base + rank] = key;
      }
    }
    __syncwarp();
  }
}

// Numeric pass with the products of a row sorted by output slot.  A group
// of W warps takes one row of C; warp w of the group owns the slots
// [w ceil(cn / W), (w + 1) ceil(cn / W)) and, in it, lane l the units
// u = l + 32 k (k < KU), unit = (slot p, block row r), summed in registers.
// The products (e, f) of the row (entries of A's row, then of B's matching
// row) are taken in their fixed enumeration order, in segments of capT:
// each product gets its slot (the position of B's column among C's sorted
// columns), products outside the warp's slots are dropped, a stable counting
// sort groups the rest by slot, and each lane adds the segment's products of
// its units in order.  Every entry of C is the same ordered sum on every run
// (no atomics on values), all lanes work even when B's rows hold a handful
// of blocks, and the shared memory per warp does not grow with the row's
// product count.  W > 1 splits long rows of C over a whole block (one group
// per block).  Rows with more slots than W warps hold or longer A rows than
// capA stay pending for the chunked kernel.
template <int BR, int BK, int BC, int KU, int W>
__global__ void __launch_bounds__(256)
    k_spgemm_numeric_seg(BsrView<double> A, BsrView<double> B, const int *rpC, const int *ciC, double *valC,
                         int *pending, int capA, int capT, int *bad) {
  constexpr int BS = BR * BC;
  constexpr int capC = (32 * KU) / BR;      // slots per warp
  constexpr int capR = capC * W;            // slots per row
  extern __shared__ int ismem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int G = wpb / W;                    // row groups per block (1 when W > 1)
  const int g = wid / W, wr = wid - g * W;
  // per group: cols (capR), pre (capA + 1); per warp: start, off, products
  const int per_group = capR + capA + 1;
  const int per_warp = 2 * capC + 1 + 4 * capT;
  int *cols = ismem + (size_t)g * per_group;
  int *pre = cols + capR;
  int *start = ismem + (size_t)G * per_group + (size_t)wid * per_warp;   // capC + 1
  int *off = start + capC + 1;    // capC
  int *pl = off + capC;           // capT: local slot of a kept segment product
  int *ee = pl + capT;            // capT: its A entry
  int *ff = ee + capT;            // capT: its B entry
  int *srt = ff + capT;           // capT: kept products sorted by slot
  const unsigned lt = (1u << lane) - 1u;
  auto sync = [&]() {
    if constexpr (W == 1) __syncwarp();
    else __syncthreads();
  };
  for (int64_t i = blockIdx.x * (int64_t)G + g; i < A.nbr; i += (int64_t)gridDim.x * G) {
    if (!pending[i]) continue;
    const int cs = rpC[i], cn = rpC[i + 1] - cs;
    const int a0 = A.rp[i], na = A.rp[i + 1] - a0;
    const int chunk = (cn + W - 1) / W;
    if (chunk > capC || na > capA) continue;
    if (wr == 0) row_product_prefix(A, B, a0, na, pre, lane);
    for (int t = wr * 32 + lane; t < cn; t += 32 * W) cols[t] = ciC[cs + t];
    sync();
    const int T = pre[na];
    const int p_lo = wr * chunk, p_n = max(0, min(cn, p_lo + chunk) - p_lo);
    double acc[KU][BC];
#pragma unroll
    for (int k = 0; k < KU; k++)
#pragma unroll
      for (int cc = 0; cc < BC; cc++) acc[k][cc] = 0.0;
    bool okp = true;
    for (int t0 = 0; t0 < T; t0 += capT) {
      const int tn = min(capT, T - t0);
      for (int t = lane; t < p_n; t += 32) {
        start[t] = 0;
        off[t] = 0;
      }
      __syncwarp();
      // slots of the segment's products; the warp keeps those in its range,
      // in enumeration order (ballot + prefix count)
      int kept = 0;
      for (int c0 = 0; c0 < tn; c0 += 32) {
        const int tl = c0 + lane;
        int e = 0, f = 0, p = -1;
        if (tl < tn) {
          const int t = t0 + tl;
          const int x = product_entry(pre, na, t);
          e = a0 + x;
          f = B.rp[A.ci[e]] + (t - pre[x]);
          p = find_sorted(cols, cn, B.ci[f]);
          if (p < 0 && tl < tn) okp = false;   // cannot happen: the symbolic pass saw every column
          p -= p_lo;
        }
        const bool keep = tl < tn && p >= 0 && p < p_n;
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int pos = kept + __popc(km & lt);
          ee[pos] = e;
          ff[pos] = f;
          pl[pos] = p;
          atomicAdd(&start[p], 1);
        }
        kept += __popc(km);
      }
      __syncwarp();
      int run = 0;
      for (int x0 = 0; x0 < p_n; x0 += 32) {
        const int x = x0 + lane;
        const int c = x < p_n ? start[x] : 0;
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        if (x < p_n) start[x] = run + inc - c;
        run += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) start[p_n] = run;
      __syncwarp();
      for (int c0 = 0; c0 < kept; c0 += 32) {
        const int tl = c0 + lane;
        const bool act = tl < kept;
        const unsigned am = __ballot_sync(0xffffffffu, act);
        int p = 0, o = 0;
        unsigned m = 0;
        if (act) {
          p = pl[tl];
          m = __match_any_sync(am, p);
          o = off[p];
          srt[start[p] + o + __popc(m & lt)] = tl;
        }
        __syncwarp();
        if (act && (m & lt) == 0) off[p] = o + __popc(m);
        __syncwarp();
      }
#pragma unroll
      for (int k = 0; k < KU; k++) {
        const int u = lane + 32 * k;
        if (u < p_n * BR) {
          const int p = u / BR, r = u - p * BR;
          const int q1 = start[p + 1];
#pragma unroll 2
          for (int q = start[p]; q < q1; q++) {
            const int tl = srt[q];
            const double *a = A.val + (int64_t)ee[tl] * BR * BK + r * BK;
            const double *b = B.val + (int64_t)ff[tl] * BK * BC;
            double av[BK];
#pragma unroll
            for (int tt = 0; tt < BK; tt++) av[tt] = a[tt];
            // straight FMA accumulation: the FP64 pipe bounds this kernel
#pragma unroll
            for (int cc = 0; cc < BC; cc++)
#pragma unroll
              for (int tt = 0; tt < BK; tt++) acc[k][cc] = fma(av[tt], b[tt * BC + cc], acc[k][cc]);
          }
        }
      }
      __syncwarp();
    }
    if (!__all_sync(0xffffffffu, okp)) {
      if (lane == 0) atomicExch(bad, 1);
    } else {
#pragma unroll
      for (int k = 0; k < KU; k++) {
        const int u = lane + 32 * k;
        if (u < p_n * BR) {
          const int p = u / BR, r = u - p * BR;
#pragma unroll
          for (int cc = 0; cc < BC; cc++) valC[(int64_t)(cs + p_lo + p) * BS + r * BC + cc] = acc[k][cc];
        }
      }
    }
    sync();
    if (wr == 0 && lane == 0) pending[i] = 0;
  }
}

// Numeric pass, one warp per row of C, FP64 work spread over all lanes.
// The row's sorted columns and accumulators live in shared memory.  The
// products (e, f) of the row (e: entry k of A's row, f: entry j of B's row
// k) are enumerated in order, in chunks; each product adds BR block-row
// contributions, and the unit (slot p of column j, block row r) is owned by
// lane (p * BR + r) mod 32.  Each lane gathers the products that touch its
// units (in enumeration order) and computes them, so every entry of C is
// summed in the same order on every run, with no atomics.
constexpr int kProdChunk = 128;

template <int BR, int BK, int BC>
__global__ void k_spgemm_numeric_sh(BsrView<double> A, BsrView<double> B, const int *rpC, const int *ciC,
                                    double *valC, const int *pending, int ulo, int ucap) {
  constexpr int BS = BR * BC;
  extern __shared__ double smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  double *acc = smem + (size_t)wid * ucap * BS;
  int *ibase = reinterpret_cast<int *>(smem + (size_t)wpb * ucap * BS);
  int *cols = ibase + (size_t)wid * (ucap + 4 * kProdChunk * BR);
  int *ch_e = cols + ucap;
  int *ch_f = ch_e + kProdChunk;
  int *ch_p = ch_f + kProdChunk;
  int *list = ch_p + kProdChunk;              // kProdChunk * BR unit-product slots
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  for (int64_t i = blockIdx.x * (int64_t)wpb + wid; i < A.nbr; i += nwarps) {
    if (!pending[i]) continue;              // done by the sorted-product kernel
    const int cs = rpC[i], cn = rpC[i + 1] - cs;
    if (cn <= ulo || cn > ucap) continue;   // another tier
    for (int t = lane; t < cn; t += 32) cols[t] = ciC[cs + t];
    for (int t = lane; t < cn * BS; t += 32) acc[t] = 0.0;
    __syncwarp();
    int cnt = 0;
    auto flush = [&]() {
      // units owned by this lane: u = p * BR + r with (u & 31) == lane
      int mine = 0;
      for (int t = 0; t < cnt; t++) {
        const int p = ch_p[t];
        if (p < 0) continue;
#pragma unroll
        for (int r = 0; r < BR; r++) mine += (((p * BR + r) & 31) == lane);
      }
      int off = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += y;
      }
      off -= mine;
      int mx = mine;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int w = off;
      for (int t = 0; t < cnt; t++) {
        const int p = ch_p[t];
        if (p < 0) continue;
#pragma unroll
        for (int r = 0; r < BR; r++)
          if (((p * BR + r) & 31) == lane) list[w++] = t * BR + r;
      }
      __syncwarp();
      for (int q = 0; q < mx; q++) {
        if (q < mine) {
          const int code = list[off + q];
          const int t = code / BR, r = code - t * BR;
          const double *a = A.val + (int64_t)ch_e[t] * BR * BK + r * BK;
          const double *b = B.val + (int64_t)ch_f[t] * BK * BC;
          double *c = acc + ch_p[t] * BS + r * BC;
          double av[BK];
#pragma unroll
          for (int tt = 0; tt < BK; tt++) av[tt] = a[tt];
#pragma unroll
          for (int cc = 0; cc < BC; cc++) {
            double v = c[cc];
#pragma unroll
            for (int tt = 0; tt < BK; tt++) v = fma(av[tt], b[tt * BC + cc], v);
            c[cc] = v;
          }
        }
      }
      __syncwarp();
      cnt = 0;
    };
    for (int e = A.rp[i]; e < A.rp[i + 1]; e++) {
      const int k = A.ci[e];
      const int f0 = B.rp[k], f1 = B.rp[k + 1];
      for (int fb = f0; fb < f1; fb += 32) {
        const int len = min(32, f1 - fb);
        if (cnt + len > kProdChunk) flush();
        if (lane < len) {
          const int f = fb + lane;
          ch_e[cnt + lane] = e;
          ch_f[cnt + lane] = f;
          ch_p[cnt + lane] = find_sorted(cols, cn, B.ci[f]);
        }
        __syncwarp();
        cnt += len;
      }
    }
    if (cnt) flush();
    for (int t = lane; t < cn * BS; t += 32) valC[(int64_t)cs * BS + t] = acc[t];
    __syncwarp();
  }
}

__global__ void k_max_pending_len(const int *rp, int n, const int *pending, int *out) {
  int m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (pending[i]) m = max(m, rp[i + 1] - rp[i]);
  atomicMax(out, m);
}

template <int BR, int BK, int BC, int KU, int W>
void launch_seg(const BsrView<double> &A, const BsrView<double> &B, Bsr<double> &C, int *pending, int *flags,
                cudaStream_t s) {
  // a block per row (W > 1) also takes long rows of A (coarse restrictions)
  const int capA = W == 1 ? 512 : 4096, capT = 192;
  const int wpb = W == 1 ? 8 : W;
  const int G = wpb / W;
  constexpr int capC = (32 * KU) / BR;
  const size_t ints = (size_t)G * (capC * W + capA + 1) + (size_t)wpb * (2 * capC + 1 + 4 * capT);
  const size_t shm = ints * sizeof(int);
  auto kern = k_spgemm_numeric_seg<BR, BK, BC, KU, W>;
  FS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  kern<<<kSMs * (W == 1 ? 8 : 2), wpb * 32, shm, s>>>(A, B, C.rp.p, C.ci.p, C.val.p, pending, capA, capT, flags);
  FS_LAUNCHED();
}

template <int BR, int BK, int BC>
void numeric(const BsrView<double> &A, const BsrView<double> &B, Bsr<double> &C, cudaStream_t s) {
  constexpr int BS = BR * BC;
  if (C.nbr == 0) return;
  DBuf<int> pending(C.nbr), flags(2);
  FS_CUDA(cudaMemsetAsync(pending.p, 1, sizeof(int) * C.nbr, s));   // nonzero = pending
  FS_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), s));
  // segmented sorted-product kernel in tiers of units per lane (KU = 4 keeps
  // the register accumulators small for the common short rows; KU = 9 takes
  // C rows up to 96 block columns per warp; eight warps per row take rows up
  // to 768 block columns): A-row entries capA, products per segment capT
  launch_seg<BR, BK, BC, 4, 1>(A, B, C, pending.p, flags.p, s);
  launch_seg<BR, BK, BC, 9, 1>(A, B, C, pending.p, flags.p, s);
  launch_seg<BR, BK, BC, 9, 8>(A, B, C, pending.p, flags.p, s);   // long rows: a block per row
  // rows beyond the tiers (very long rows of A or many products): longest C row among them
  k_max_pending_len<<<blocks_for(C.nbr, 256, kSMs * 4), 256, 0, s>>>(C.rp.p, C.nbr, pending.p, flags.p + 1);
  FS_LAUNCHED();
  int hf[2] = {0, 0};
  FS_CUDA(cudaMemcpyAsync(hf, flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!hf[0], FC_INTERNAL, "spgemm: a product column is missing from the symbolic pattern");
  const int umax = hf[1];
  if (umax == 0) return;
  // the chunked kernel, in tiers of C-row length so that short rows run at
  // higher occupancy: per warp, ucap slots (accumulator + column) and the
  // product chunk
  const size_t per_slot = BS * sizeof(double) + sizeof(int);
  const size_t fixed = (size_t)4 * kProdChunk * BR * sizeof(int);
  const int ctiers[3] = {64, 256, kListCap};
  FS_REQUIRE(umax <= kListCap, FC_INTERNAL, "spgemm: product row longer than the symbolic pass allows");
  int ulo = 0;
  for (int t = 0; t < 3 && ulo < umax; t++) {
    const int ucap = ctiers[t];
    int wpb = 8;
    while (wpb > 1 && (size_t)wpb * (ucap * per_slot + fixed) > 200 * 1024) wpb >>= 1;
    const size_t shm = (size_t)wpb * (ucap * per_slot + fixed);
    auto kern = k_spgemm_numeric_sh<BR, BK, BC>;
    FS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    kern<<<kSMs * 8, wpb * 32, shm, s>>>(A, B, C.rp.p, C.ci.p, C.val.p, pending.p, ulo, ucap);
    FS_LAUNCHED();
    ulo = ucap;
  }
}

}  // namespace

void spgemm_numeric(const BsrView<double> &A, const BsrView<double> &B, Bsr<double> &C, cudaStream_t s) {
  FS_REQUIRE(A.bc == B.br && A.nbc == B.nbr && C.nbr == A.nbr && C.nbc == B.nbc && C.br == A.br && C.bc == B.bc,
             FC_BAD_ARG, "spgemm_numeric: shape mismatch");
  if (C.nnzb == 0) return;
  const int sh = A.br * 100 + A.bc * 10 + B.bc;
  switch (sh) {
    case 333: numeric<3, 3, 3>(A, B, C, s); break;
    case 313: numeric<3, 1, 3>(A, B, C, s); break;
    case 111: numeric<1, 1, 1>(A, B, C, s); break;
    case 331: numeric<3, 3, 1>(A, B, C, s); break;
    case 133: numeric<1, 3, 3>(A, B, C, s); break;
    default: throw Error(FC_BAD_ARG, "spgemm: unsupported block shapes");
  }
}

namespace {
__global__ void k_diff_int(const int *a, const int *b, int64_t n, int *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) {
      atomicExch(out, 1);
      return;
    }
}
__global__ void k_diff_bits(const unsigned long long *a, const unsigned long long *b, int64_t n, int *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != b[i]) {
      atomicExch(out, 1);
      return;
    }
}
}  // namespace

namespace {
// row pointers: rp[0] = 0, non-decreasing, rp[nbr] = nnzb (flag bit 1)
__global__ void k_check_rp(const int *rp, int nbr, int64_t nnzb, int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int v = rp[i];
    bool ok = v >= 0 && (int64_t)v <= nnzb;
    if (i == 0) ok = ok && v == 0;
    if (i == nbr) ok = ok && (int64_t)v == nnzb;
    if (i < nbr) ok = ok && rp[i + 1] >= v;
    if (!ok) atomicOr(flag, 1);
  }
}
// columns within [0, nbc), strictly increasing in each row (flag bit 2);
// only run once the row pointers passed
__global__ void k_check_ci(const int *rp, const int *ci, int nbr, int nbc, int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int prev = -1;
    for (int e = rp[i]; e < rp[i + 1]; e++) {
      const int c = ci[e];
      if (c <= prev || c >= nbc) {
        atomicOr(flag, 2);
        break;
      }
      prev = c;
    }
  }
}
}  // namespace

int check_structure(const BsrView<double> &A, cudaStream_t s) {
  DBuf<int> f(1);
  FS_CUDA(cudaMemsetAsync(f.p, 0, sizeof(int), s));
  k_check_rp<<<blocks_for((int64_t)A.nbr + 1, 256, kSMs * 8), 256, 0, s>>>(A.rp, A.nbr, A.nnzb, f.p);
  FS_LAUNCHED();
  int h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, f.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  if (h) return 1;
  if (A.nbr > 0 && A.nnzb > 0) {
    k_check_ci<<<blocks_for(A.nbr, 128, kSMs * 16), 128, 0, s>>>(A.rp, A.ci, A.nbr, A.nbc, f.p);
    FS_LAUNCHED();
    FS_CUDA(cudaMemcpyAsync(&h, f.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
  }
  return h;
}

bool same_values(const double *a, const double *b, int64_t n, cudaStream_t s) {
  if (n <= 0) return true;
  DBuf<int> d(1);
  FS_CUDA(cudaMemsetAsync(d.p, 0, sizeof(int), s));
  k_diff_bits<<<blocks_for(n, 256, kSMs * 8), 256, 0, s>>>(reinterpret_cast<const unsigned long long *>(a),
                                                           reinterpret_cast<const unsigned long long *>(b), n, d.p);
  FS_LAUNCHED();
  int h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, d.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  return h == 0;
}

bool same_pattern(const BsrView<double> &A, const BsrView<double> &B, cudaStream_t s) {
  if (A.nbr != B.nbr || A.nbc != B.nbc || A.br != B.br || A.bc != B.bc || A.nnzb != B.nnzb) return false;
  DBuf<int> d(1);
  FS_CUDA(cudaMemsetAsync(d.p, 0, sizeof(int), s));
  k_diff_int<<<blocks_for((int64_t)A.nbr + 1, 256, kSMs * 8), 256, 0, s>>>(A.rp, B.rp, (int64_t)A.nbr + 1, d.p);
  FS_LAUNCHED();
  if (A.nnzb) {
    k_diff_int<<<blocks_for(A.nnzb, 256, kSMs * 8), 256, 0, s>>>(A.ci, B.ci, A.nnzb, d.p);
    FS_LAUNCHED();
  }
  int h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, d.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  return h == 0;
}

Bsr<double> spgemm(const BsrView<double> &A, const BsrView<double> &B, cudaStream_t s) {
  FS_REQUIRE(A.bc == B.br && A.nbc == B.nbr, FC_BAD_ARG, "spgemm: shape mismatch");
  Bsr<double> C;
  C.shape(A.nbr, B.nbc, A.br, B.bc);
  C.rp.alloc(A.nbr + 1);
  DBuf<int> cnt(A.nbr + 1), ovf(1);
  FS_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), s));
  FS_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (A.nbr + 1), s));
  const int grid = kSMs * 8;
  PhaseTimer pt(g_verbose > 1, s, "spgemm");
  if (A.nbr > 0) {
    k_spgemm_symbolic<<<grid, kWarpsPerBlock * 32, 0, s>>>(A, B, 0, cnt.p, nullptr, nullptr, ovf.p);
    FS_LAUNCHED();
  }
  pt.mark("symbolic count");
  int64_t nnz = exclusive_scan(cnt.p, C.rp.p, A.nbr, s);
  int hovf = 0;
  FS_CUDA(cudaMemcpy(&hovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost));
  FS_REQUIRE(!hovf, FC_INTERNAL, "spgemm: a product row has more than 768 block columns");
  C.nnzb = nnz;
  C.ci.alloc(nnz);
  C.val.alloc(nnz * C.br * C.bc);
  if (nnz == 0) return C;
  pt.mark("scan + alloc");
  k_spgemm_symbolic<<<grid, kWarpsPerBlock * 32, 0, s>>>(A, B, 1, nullptr, C.rp.p, C.ci.p, ovf.p);
  FS_LAUNCHED();
  pt.mark("symbolic fill");
  const int sh = A.br * 100 + A.bc * 10 + B.bc;
  switch (sh) {
    case 333: numeric<3, 3, 3>(A, B, C, s); break;
    case 313: numeric<3, 1, 3>(A, B, C, s); break;
    case 111: numeric<1, 1, 1>(A, B, C, s); break;
    case 331: numeric<3, 3, 1>(A, B, C, s); break;
    case 133: numeric<1, 3, 3>(A, B, C, s); break;
    default: throw Error(FC_BAD_ARG, "spgemm: unsupported block shapes");
  }
  pt.mark("numeric");
  if (g_verbose > 1)
    fprintf(stderr, "[fracsolve] spgemm %d x %d blocks (%dx%d * %dx%d): A %lld, B %lld, C %lld blocks\n", A.nbr, B.nbc,
            A.br, A.bc, B.br, B.bc, (long long)A.nnzb, (long long)B.nnzb, (long long)nnz);
  FS_CUDA(cudaStreamSynchronize(s));
  return C;
}

// ============================================================ sparse add
namespace {
__global__ void k_spadd(BsrView<double> A, BsrView<double> B, double alpha, double beta, int pass,
                        int *cnt, const int *rpC, int *ciC, double *valC) {
  const int bs = A.br * A.bc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = A.rp[i], ae = A.rp[i + 1], b = B.rp[i], be = B.rp[i + 1];
    int n = 0;
    int o = pass ? rpC[i] : 0;
    while (a < ae || b < be) {
      int ca = a < ae ? A.ci[a] : INT32_MAX;
      int cb = b < be ? B.ci[b] : INT32_MAX;
      int c = ca < cb ? ca : cb;
      if (pass) {
        ciC[o + n] = c;
        double *dst = valC + (int64_t)(o + n) * bs;
        for (int q = 0; q < bs; q++) {
          double v = 0.0;
          if (ca == c) v += alpha * A.val[(int64_t)a * bs + q];
          if (cb == c) v += beta * B.val[(int64_t)b * bs + q];
          dst[q] = v;
        }
      }
      if (ca == c) a++;
      if (cb == c) b++;
      n++;
    }
    if (!pass) cnt[i] = n;
  }
}
}  // namespace

Bsr<double> spadd(const BsrView<double> &A, const BsrView<double> &B, double alpha, double beta,
                  cudaStream_t s) {
  FS_REQUIRE(A.nbr == B.nbr && A.nbc == B.nbc && A.br == B.br && A.bc == B.bc, FC_BAD_ARG,
             "spadd: shape mismatch");
  Bsr<double> C;
  C.shape(A.nbr, A.nbc, A.br, A.bc);
  C.rp.alloc(A.nbr + 1);
  DBuf<int> cnt(A.nbr + 1);
  const int grid = blocks_for(A.nbr, 128, kSMs * 8);
  if (A.nbr > 0) {
    k_spadd<<<grid, 128, 0, s>>>(A, B, alpha, beta, 0, cnt.p, nullptr, nullptr, nullptr);
    FS_LAUNCHED();
  }
  int64_t nnz = exclusive_scan(cnt.p, C.rp.p, A.nbr, s);
  C.nnzb = nnz;
  C.ci.alloc(nnz);
  C.val.alloc(nnz * C.br * C.bc);
  if (nnz) {
    k_spadd<<<grid, 128, 0, s>>>(A, B, alpha, beta, 1, nullptr, C.rp.p, C.ci.p, C.val.p);
    FS_LAUNCHED();
  }
  FS_CUDA(cudaStreamSynchronize(s));
  return C;
}

// ============================================================ copies
namespace {
template <typename TO, typename TI>
__global__ void k_cast_vals(TO *o, const TI *i, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    o[k] = (TO)i[k];
}
}  // namespace

template <typename TO, typename TI>
Bsr<TO> copy_cast(const BsrView<TI> &A, cudaStream_t s) {
  Bsr<TO> C;
  C.shape(A.nbr, A.nbc, A.br, A.bc);
  C.nnzb = A.nnzb;
  C.rp.alloc(A.nbr + 1);
  C.ci.alloc(A.nnzb);
  C.val.alloc(A.nnzb * A.br * A.bc);
  FS_CUDA(cudaMemcpyAsync(C.rp.p, A.rp, sizeof(int) * (A.nbr + 1), cudaMemcpyDeviceToDevice, s));
  if (A.nnzb) {
    FS_CUDA(cudaMemcpyAsync(C.ci.p, A.ci, sizeof(int) * A.nnzb, cudaMemcpyDeviceToDevice, s));
    int64_t n = A.nnzb * A.br * A.bc;
    k_cast_vals<TO, TI><<<blocks_for(n, 256, kSMs * 16), 256, 0, s>>>(C.val.p, A.val, n);
    FS_LAUNCHED();
  }
  return C;
}
template Bsr<float> copy_cast<float, double>(const BsrView<double> &, cudaStream_t);
template Bsr<double> copy_cast<double, double>(const BsrView<double> &, cudaStream_t);

// ============================================================ sliced ELL
namespace {
__global__ void k_sell_width(BsrView<double> A, int nslice, int *w) {
  for (int64_t sl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sl < nslice;
       sl += (int64_t)gridDim.x * blockDim.x) {
    int m = 0;
    for (int r = 0; r < kSellH; r++) {
      int64_t row = sl * kSellH + r;
      if (row >= A.nbr) break;
      int len = A.rp[row + 1] - A.rp[row];
      m = len > m ? len : m;
    }
    w[sl] = m;
  }
}

__global__ void k_to_i64(const int *in, int64_t *out, int n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

template <typename T>
__global__ void k_sell_fill(BsrView<double> A, int nslice, const int64_t *sp, int *ci, T *val) {
  const int bs = A.br * A.bc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nslice * kSellH;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = t / kSellH;
    const int lane = (int)(t % kSellH);
    const int64_t s0 = sp[sl], w = sp[sl + 1] - s0;
    const bool real = t < A.nbr;
    const int b0 = real ? A.rp[t] : 0;
    const int len = real ? A.rp[t + 1] - b0 : 0;
    for (int64_t k = 0; k < w; k++) {
      const int64_t slot = s0 + k;
      if (k < len) {
        ci[slot * kSellH + lane] = A.ci[b0 + k];
        for (int q = 0; q < bs; q++) val[(slot * bs + q) * kSellH + lane] = (T)A.val[(int64_t)(b0 + k) * bs + q];
      } else {
        ci[slot * kSellH + lane] = 0;
        for (int q = 0; q < bs; q++) val[(slot * bs + q) * kSellH + lane] = T(0);
      }
    }
  }
}
}  // namespace

template <typename T>
Sell<T> to_sell(const BsrView<double> &A, cudaStream_t s) {
  Sell<T> S;
  S.nbr = A.nbr; S.nbc = A.nbc; S.br = A.br; S.bc = A.bc; S.nnzb = A.nnzb;
  S.nslice = (A.nbr + kSellH - 1) / kSellH;
  S.sp.alloc(S.nslice + 1);
  if (S.nslice == 0) {
    FS_CUDA(cudaMemsetAsync(S.sp.p, 0, sizeof(int64_t), s));
    return S;
  }
  DBuf<int> w(S.nslice + 1), wp(S.nslice + 1);
  k_sell_width<<<blocks_for(S.nslice, 128, kSMs * 8), 128, 0, s>>>(A, S.nslice, w.p);
  FS_LAUNCHED();
  S.slots = exclusive_scan(w.p, wp.p, S.nslice, s);
  k_to_i64<<<blocks_for(S.nslice + 1, 256, kSMs * 4), 256, 0, s>>>(wp.p, S.sp.p, S.nslice);
  FS_LAUNCHED();
  S.ci.alloc(S.slots * kSellH);
  S.val.alloc(S.slots * kSellH * A.br * A.bc);
  if (S.slots) {
    k_sell_fill<T><<<blocks_for((int64_t)S.nslice * kSellH, 128, kSMs * 16), 128, 0, s>>>(A, S.nslice, S.sp.p, S.ci.p,
                                                                                       S.val.p);
    FS_LAUNCHED();
  }
  return S;
}
template Sell<float> to_sell<float>(const BsrView<double> &, cudaStream_t);
template Sell<double> to_sell<double>(const BsrView<double> &, cudaStream_t);

Bsr<double> upload_bsr(int nbr, int nbc, int br, int bc, int64_t nnzb, const int *rp_dev,
                       const int *ci_dev, const double *val_dev, cudaStream_t s) {
  BsrView<double> v;
  v.nbr = nbr; v.nbc = nbc; v.br = br; v.bc = bc; v.nnzb = nnzb;
  v.rp = rp_dev; v.ci = ci_dev; v.val = val_dev;
  return copy_cast<double, double>(v, s);
}

void download_bsr(const BsrView<double> &A, std::vector<int> &rp, std::vector<int> &ci,
                  std::vector<double> &val, cudaStream_t s) {
  rp.resize(A.nbr + 1);
  ci.resize(A.nnzb);
  val.resize(A.nnzb * A.br * A.bc);
  FS_CUDA(cudaMemcpyAsync(rp.data(), A.rp, sizeof(int) * (A.nbr + 1), cudaMemcpyDeviceToHost, s));
  if (A.nnzb) {
    FS_CUDA(cudaMemcpyAsync(ci.data(), A.ci, sizeof(int) * A.nnzb, cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaMemcpyAsync(val.data(), A.val, sizeof(double) * val.size(), cudaMemcpyDeviceToHost, s));
  }
  FS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fs
