// Setup-phase sparse kernels: transpose, block SpGEMM, sparse add.
#include <cstdlib>

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
constexpr int64_t kStashMax = (int64_t)1 << 30;   // stash entries of the one-enumeration symbolic pass, at most

struct WarpHash {
  int *keys;   // kHashCap
  int *list;   // kListCap
  int *count;  // 1
  int mask;    // slots in use - 1 (a power of two minus one)
};

// use the smallest power-of-two table of at least 2 n slots (n keys at most;
// 32 at least, kHashCap at most) and empty it
__device__ inline void hash_clear(WarpHash &h, int lane, int n) {
  int cap = 32;
  while (cap < 2 * n && cap < kHashCap) cap <<= 1;
  h.mask = cap - 1;
  for (int k = lane; k < cap; k += 32) h.keys[k] = -1;
  if (lane == 0) *h.count = 0;
  __syncwarp();
}

// returns false on overflow
__device__ inline bool hash_insert(WarpHash &h, int key) {
  unsigned slot = ((unsigned)key * 2654435761u) & h.mask;
  for (int probe = 0; probe <= h.mask; probe++) {
    int old = atomicCAS(h.keys + slot, -1, key);
    if (old == -1) {
      int pos = atomicAdd(h.count, 1);
      if (pos >= kListCap) return false;
      h.list[pos] = key;
      return true;
    }
    if (old == key) return true;
    slot = (slot + 1) & h.mask;
  }
  return false;
}

// Prefix of the B-row lengths over the row of A (a0, na): pre[x] = products
// of entries 0..x-1, pre[na] = T (returned to every lane).
template <typename TV>
__device__ inline int row_product_prefix(const BsrView<TV> &A, const BsrView<TV> &B, int a0, int na,
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

// pass 0: count unique columns per row and, when stash is given, keep them
// (unsorted) at stash + soff[i]; pass 1: write sorted columns.  The products
// of a row are enumerated flat (all lanes busy even when the rows of B are
// short); rows of A longer than kSymPre take the entry-by-entry loop.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_spgemm_symbolic(BsrView<double> A, BsrView<double> B, int pass, int *cnt, const int *rpC,
                      int *ciC, int *overflow, int *stash = nullptr, const int *soff = nullptr) {
  __shared__ int s_keys[kWarpsPerBlock][kHashCap];
  __shared__ int s_list[kWarpsPerBlock][kListCap];
  __shared__ int s_pre[kWarpsPerBlock][kSymPre + 1];
  __shared__ int s_kb[kWarpsPerBlock][kSymPre];
  __shared__ int s_cnt[kWarpsPerBlock];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpHash h{s_keys[wid], s_list[wid], &s_cnt[wid], kHashCap - 1};
  int *pre = s_pre[wid], *kb = s_kb[wid];
  const int64_t nwarps = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t i = blockIdx.x * (int64_t)kWarpsPerBlock + wid; i < A.nbr; i += nwarps) {
    bool ok = true;
    const int a0 = A.rp[i], na = A.rp[i + 1] - a0;
    if (na <= kSymPre) {
      const int T = row_product_prefix(A, B, a0, na, pre, lane);
      for (int x = lane; x < na; x += 32) kb[x] = B.rp[A.ci[a0 + x]];
      hash_clear(h, lane, T);
      // four products per lane at a time: their column loads issue together
      for (int t0 = 0; t0 < T; t0 += 128) {
        int cv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int t = t0 + u * 32 + lane;
          cv[u] = -1;
          if (t < T) {
            const int x = product_entry(pre, na, t);
            cv[u] = B.ci[kb[x] + (t - pre[x])];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
          if (cv[u] >= 0) ok &= hash_insert(h, cv[u]);
      }
    } else {
      hash_clear(h, lane, kHashCap);
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
      if (stash)
        for (int a = lane; a < u; a += 32) stash[soff[i] + a] = h.list[a];
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

// stash capacity of each row of C = A B: its product count, at most kListCap
__global__ void k_stash_cap(BsrView<double> A, BsrView<double> B, int *cap) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < A.nbr; i += nw) {
    int t = 0;
    for (int e = A.rp[i] + lane; e < A.rp[i + 1]; e += 32) {
      const int k = A.ci[e];
      t += B.rp[k + 1] - B.rp[k];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) cap[i] = min(t, kListCap);
  }
}

// columns of row i of C: its stashed unique columns, sorted by rank
__global__ void k_stash_sort(int nbr, const int *stash, const int *soff, const int *rpC, int *ciC) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nbr; i += nw) {
    const int base = rpC[i], u = rpC[i + 1] - base;
    const int *l = stash + soff[i];
    for (int a = lane; a < u; a += 32) {
      const int key = l[a];
      int rank = 0;
      for (int b = 0; b < u; b++) rank += (l[b] < key);
      ciC[base + rank] = key;
    }
  }
}

// Numeric pass with the products of a row sorted by output slot and split
// evenly over the lanes.  One warp per row of C (the rows of a length class,
// from a list); the row's slot sums live in shared memory.  The row's
// products (e, f) (entries of A's row, then of B's matching row) are taken
// in their fixed enumeration order in segments of capT (a multiple of
// kSegT, by row class); each gets its slot
// (the position of B's column among C's sorted columns) and a stable
// counting sort groups the segment by slot.  The sorted list is then cut
// into 32 equal runs, one per lane: a lane adds its run's products in order
// into a register block, starting from the slot's sum so far when the slot
// begins in its run (the lane then owns it) and from zero when the slot
// continues from the lane before; the owner then adds those continuations
// in lane order.  Every FP64 instruction thus runs on a full warp (the FP64
// pipe executes a warp instruction whole, active lanes or not), and every
// entry of C is the same ordered sum on every run, with no value atomics.
constexpr int kSegT = 192;   // products per segment of the numeric pass

// A share of one row's products, [t_lo, t_hi) in enumeration order, summed
// into scratch + soff (soff >= 0: a row split over several warps) or into
// the row of C itself (soff < 0).
struct SpgemmTask {
  int row, t_lo, t_hi;
  int64_t soff;
};

template <typename T, int BR, int BK, int BC, bool GS>
__global__ void __launch_bounds__(256)
    k_spgemm_numeric_mp(BsrView<T> A, BsrView<T> B, const int *rpC, const int *ciC, T *valC,
                        const int *rows, const int *nrows, const SpgemmTask *tasks, T *scratch, int capA,
                        int capC, int capT, int *bad) {
  constexpr int BS = BR * BC, AS = BR * BK, BB = BK * BC, kPL = kSegT / 32;
  extern __shared__ double dsm_raw[];
  T *dsm = reinterpret_cast<T *>(dsm_raw);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int dw = (GS ? 0 : capC) + 32;                   // values per warp, in blocks
  T *carry = dsm + (size_t)wid * dw * BS;                 // 32 continuation sums
  int *cols = reinterpret_cast<int *>(dsm + (size_t)wpb * dw * BS) +
              (size_t)wid * (3 * capC + 2 * capA + 2 + 4 * capT);
  int *pre = cols + capC;          // capA + 1
  int *kb = pre + capA + 1;        // capA: start of B's row for each A entry
  int *start = kb + capA;          // capC + 1
  int *off = start + capC + 1;     // capC
  int *pl = off + capC;            // capT: slot of a segment product
  int *ee = pl + capT;             // capT: its A entry
  int *ff = ee + capT;             // capT: its B entry
  int *srt = ff + capT;            // capT: the products sorted by slot
  const unsigned lt = (1u << lane) - 1u;
  const int n = *nrows;
  for (int w = blockIdx.x * wpb + wid; w < n; w += gridDim.x * wpb) {
    const SpgemmTask tk = tasks ? tasks[w] : SpgemmTask{rows[w], 0, INT32_MAX, -1};
    const int i = tk.row;
    const int cs = rpC[i], p_n = rpC[i + 1] - cs;
    const int a0 = A.rp[i], na = A.rp[i + 1] - a0;
    // the slot sums: in shared memory, or (long rows) the row of C itself or
    // this task's share of the scratch
    T *sums = !GS ? carry + 32 * BS : tk.soff >= 0 ? scratch + tk.soff : valC + (int64_t)cs * BS;
    row_product_prefix(A, B, a0, na, pre, lane);
    for (int x = lane; x < na; x += 32) kb[x] = B.rp[A.ci[a0 + x]];
    for (int t = lane; t < p_n; t += 32) cols[t] = ciC[cs + t];
    __syncwarp();
    const int tend = min(pre[na], tk.t_hi);
    for (int x = lane; x < p_n * BS; x += 32) sums[x] = T(0);
    bool okp = true;
    for (int t0 = tk.t_lo; t0 < tend; t0 += capT) {
      const int tn = min(capT, tend - t0);
      for (int t = lane; t < p_n; t += 32) {
        start[t] = 0;
        off[t] = 0;
      }
      __syncwarp();
      // the segment's products, kSegT at a time: kPL per lane, their loads
      // issued together
      for (int c0 = 0; c0 < tn; c0 += kSegT) {
        int ev[kPL], fv[kPL], cv[kPL];
#pragma unroll
        for (int u = 0; u < kPL; u++) {
          const int tl = c0 + u * 32 + lane;
          ev[u] = 0;
          fv[u] = 0;
          if (tl < tn) {
            const int t = t0 + tl;
            const int x = product_entry(pre, na, t);
            ev[u] = a0 + x;
            fv[u] = kb[x] + (t - pre[x]);
          }
        }
#pragma unroll
        for (int u = 0; u < kPL; u++) cv[u] = c0 + u * 32 + lane < tn ? B.ci[fv[u]] : 0;
#pragma unroll
        for (int u = 0; u < kPL; u++) {
          const int tl = c0 + u * 32 + lane;
          if (tl < tn) {
            int p = find_sorted(cols, p_n, cv[u]);
            if (p < 0) {   // cannot happen: the symbolic pass saw every column
              okp = false;
              p = 0;
            }
            ee[tl] = ev[u];
            ff[tl] = fv[u];
            pl[tl] = p;
            atomicAdd(&start[p], 1);
          }
        }
      }
      const int kept = tn;
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
      // this lane's run of the sorted products
      const int q_lo = (lane * kept) >> 5, q_hi = ((lane + 1) * kept) >> 5;
      int cur = -1;
      bool own = false;
      if (q_lo < q_hi) {
        T acc[BS], av[AS], bv[BB], an[AS], bn[BB];
        int tl = srt[q_lo];
        cur = pl[tl];
        own = start[cur] == q_lo;
#pragma unroll
        for (int x = 0; x < BS; x++) acc[x] = own ? sums[cur * BS + x] : T(0);
        {
          const T *a = A.val + (int64_t)ee[tl] * AS, *b = B.val + (int64_t)ff[tl] * BB;
#pragma unroll
          for (int x = 0; x < AS; x++) av[x] = a[x];
#pragma unroll
          for (int x = 0; x < BB; x++) bv[x] = b[x];
        }
        for (int q = q_lo; q < q_hi; q++) {
          int tn2 = 0;
          if (q + 1 < q_hi) {   // fetch the next product's blocks while this one is summed
            tn2 = srt[q + 1];
            const T *a = A.val + (int64_t)ee[tn2] * AS, *b = B.val + (int64_t)ff[tn2] * BB;
#pragma unroll
            for (int x = 0; x < AS; x++) an[x] = a[x];
#pragma unroll
            for (int x = 0; x < BB; x++) bn[x] = b[x];
          }
          const int p = pl[tl];
          if (p != cur) {   // a new slot begins here: this lane owns it
            if (own) {
#pragma unroll
              for (int x = 0; x < BS; x++) sums[cur * BS + x] = acc[x];
            } else {
#pragma unroll
              for (int x = 0; x < BS; x++) carry[lane * BS + x] = acc[x];
            }
            cur = p;
            own = true;
#pragma unroll
            for (int x = 0; x < BS; x++) acc[x] = sums[cur * BS + x];
          }
#pragma unroll
          for (int r = 0; r < BR; r++)
#pragma unroll
            for (int k = 0; k < BK; k++)
#pragma unroll
              for (int c = 0; c < BC; c++) acc[r * BC + c] = fma(av[r * BK + k], bv[k * BC + c], acc[r * BC + c]);
          tl = tn2;
#pragma unroll
          for (int x = 0; x < AS; x++) av[x] = an[x];
#pragma unroll
          for (int x = 0; x < BB; x++) bv[x] = bn[x];
        }
        if (own) {
#pragma unroll
          for (int x = 0; x < BS; x++) sums[cur * BS + x] = acc[x];
        } else {
#pragma unroll
          for (int x = 0; x < BS; x++) carry[lane * BS + x] = acc[x];
        }
      }
      __syncwarp();
      // the owner of the run's last slot adds the continuations of the
      // following lanes, in lane order
      if (own) {
        const int end = start[cur + 1];
        for (int l = lane + 1; l < 32; l++) {
          const int lo = (l * kept) >> 5;
          if (lo >= end) break;
          if (((l + 1) * kept) >> 5 > lo) {
#pragma unroll
            for (int x = 0; x < BS; x++) sums[cur * BS + x] += carry[l * BS + x];
          }
        }
      }
      __syncwarp();
    }
    if (!__all_sync(0xffffffffu, okp)) {
      if (lane == 0) atomicExch(bad, 1);
    } else if (!GS) {
      for (int x = lane; x < p_n * BS; x += 32) valC[(int64_t)cs * BS + x] = sums[x];
    }
    __syncwarp();
  }
}

// Length classes of the rows of C for the numeric pass: class c takes rows
// with at most caps[c] columns and an A row of at most capa[c] entries;
// rows beyond the last class stay pending for the chunked kernel.
struct RowClasses {
  int n;
  int caps[3], capa[3];
};

__global__ void k_classify_rows(const int *rpA, const int *rpC, int nbr, RowClasses rc, int *lists, int *counts,
                                int *pending) {
  const int lane = threadIdx.x & 31;
  // whole warps iterate (the grid stride is a multiple of 32); the lanes of
  // one class take their list positions with one atomic
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < nbr;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + lane;
    int c = rc.n + 1;   // no row
    if (i < nbr) {
      const int cn = rpC[i + 1] - rpC[i], na = rpA[i + 1] - rpA[i];
      c = 0;
      while (c < rc.n && (cn > rc.caps[c] || na > rc.capa[c])) c++;
    }
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (c < rc.n && lane == leader) base = atomicAdd(counts + c, __popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (c < rc.n) {
      lists[(int64_t)c * nbr + base + __popc(same & ((1u << lane) - 1u))] = (int)i;
      pending[i] = 0;
    } else if (i < nbr) {
      pending[i] = 1;
    }
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

template <typename T, int BR, int BK, int BC>
__global__ void k_spgemm_numeric_sh(BsrView<T> A, BsrView<T> B, const int *rpC, const int *ciC,
                                    T *valC, const int *pending, int ulo, int ucap) {
  constexpr int BS = BR * BC;
  extern __shared__ double smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  T *acc = smem + (size_t)wid * ucap * BS;
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
    for (int t = lane; t < cn * BS; t += 32) acc[t] = T(0);
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
          const T *a = A.val + (int64_t)ch_e[t] * BR * BK + r * BK;
          const T *b = B.val + (int64_t)ch_f[t] * BK * BC;
          T *c = acc + ch_p[t] * BS + r * BC;
          T av[BK];
#pragma unroll
          for (int tt = 0; tt < BK; tt++) av[tt] = a[tt];
#pragma unroll
          for (int cc = 0; cc < BC; cc++) {
            T v = c[cc];
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

// products and columns of the listed rows of C = A B
template <typename T>
__global__ void k_row_info(BsrView<T> A, BsrView<T> B, const int *rpC, const int *rows, int n,
                           int *nprod, int *pn) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < n; w += nw) {
    const int i = rows[w];
    int t = 0;
    for (int e = A.rp[i] + lane; e < A.rp[i + 1]; e += 32) {
      const int k = A.ci[e];
      t += B.rp[k + 1] - B.rp[k];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      nprod[w] = t;
      pn[w] = rpC[i + 1] - rpC[i];
    }
  }
}

struct SplitRow {
  int row, nt, pn;
  int64_t soff;
};

// a row split over nt tasks: its sums, added in task order
template <typename T>
__global__ void k_sum_split(const SplitRow *sr, int n, const int *rpC, const T *scratch, int bs,
                            T *valC) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < n; w += nw) {
    const SplitRow r = sr[w];
    const int64_t len = (int64_t)r.pn * bs;
    for (int64_t x = lane; x < len; x += 32) {
      T v = scratch[r.soff + x];
      for (int k = 1; k < r.nt; k++) v += scratch[r.soff + k * len + x];
      valC[(int64_t)rpC[r.row] * bs + x] = v;
    }
  }
}

template <typename T, int BR, int BK, int BC, bool GS>
void launch_mp(const BsrView<T> &A, const BsrView<T> &B, Bsr<T> &C, const int *rows,
               const int *nrows, const SpgemmTask *tasks, T *scratch, int capC, int capA, int capT,
               int *flags, cudaStream_t s) {
  // shared memory per warp; up to eight warps per block, as many blocks per SM as fit
  const size_t per_warp = (size_t)((GS ? 0 : capC) + 32) * BR * BC * sizeof(T) +
                          (size_t)(3 * capC + 2 * capA + 2 + 4 * capT) * sizeof(int);
  const size_t budget = 225 * 1024;
  FS_REQUIRE(per_warp <= budget, FC_INTERNAL, "spgemm: row class does not fit in shared memory");
  const int wpb = (int)std::min<size_t>(8, budget / per_warp);
  const size_t shm = per_warp * wpb;
  const int per_sm = (int)std::min<size_t>(4, std::max<size_t>(1, budget / shm));
  auto kern = k_spgemm_numeric_mp<T, BR, BK, BC, GS>;
  FS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  kern<<<kSMs * per_sm, wpb * 32, shm, s>>>(A, B, C.rp.p, C.ci.p, C.val.p, rows, nrows, tasks, scratch, capA, capC,
                                            capT, flags);
  FS_LAUNCHED();
}

constexpr int kTaskT = 8 * kSegT;                  // products per task of a split row, at least
constexpr size_t kSplitScratch = (size_t)512 << 20;   // bytes of partial sums, at most

template <typename T, int BR, int BK, int BC>
void numeric(const BsrView<T> &A, const BsrView<T> &B, Bsr<T> &C, cudaStream_t s) {
  constexpr int BS = BR * BC;
  if (C.nbr == 0) return;
  // three length classes of C rows (columns, A-row entries): short rows sum
  // in shared memory at two blocks per SM; medium and long rows sum in the
  // row of C itself, which keeps eight or more warps per SM.  Long rows with
  // many products are split into tasks of kTaskT or more products, summed
  // apart and added in task order.
  RowClasses rc{3, {64, 160, 768}, {256, 512, 1024}};
  // test hook, compiled only into the test build (FS_TEST_HOOKS):
  // FS_SPGEMM_FORCE_LONG=<products> sends every row that fits the long class
  // there and splits rows into tasks of that many products; -1 leaves every
  // row to the chunked kernel that takes rows beyond the classes.  Small
  // problems then exercise the paths large ones take.  The product library
  // reads no environment variable.
  int64_t task_min = kTaskT;
#ifdef FS_TEST_HOOKS
  if (const char *ev = std::getenv("FS_SPGEMM_FORCE_LONG")) {
    const long v = std::strtol(ev, nullptr, 10);
    if (v > 0) {
      rc.caps[0] = rc.caps[1] = -1;
      task_min = v;
    } else if (v == -1) {
      rc.caps[0] = rc.caps[1] = rc.caps[2] = -1;
    }
  }
#endif
  DBuf<int> pending(C.nbr), flags(2), lists((size_t)rc.n * C.nbr), counts(rc.n);
  FS_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), s));
  FS_CUDA(cudaMemsetAsync(counts.p, 0, rc.n * sizeof(int), s));
  k_classify_rows<<<blocks_for(C.nbr, 256, kSMs * 8), 256, 0, s>>>(A.rp, C.rp.p, C.nbr, rc, lists.p, counts.p,
                                                                    pending.p);
  FS_LAUNCHED();
  // segments of kSegT products in every class (longer segments for the
  // longer rows, 768 and 1536 products, were slower at 128^3: fewer warps
  // per SM)
  launch_mp<T, BR, BK, BC, false>(A, B, C, lists.p, counts.p, nullptr, nullptr, rc.caps[0], rc.capa[0], kSegT,
                               flags.p, s);
  launch_mp<T, BR, BK, BC, true>(A, B, C, lists.p + C.nbr, counts.p + 1, nullptr, nullptr, rc.caps[1], rc.capa[1],
                              kSegT, flags.p, s);
  int hc[3] = {0, 0, 0};
  FS_CUDA(cudaMemcpyAsync(hc, counts.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  const int n2 = hc[2];
  DBuf<SpgemmTask> dtasks;
  DBuf<SplitRow> dsplit;
  DBuf<T> scratch;
  DBuf<int> ntask;
  int nsplit = 0;
  if (n2 > 0) {
    const int *rows2 = lists.p + (size_t)2 * C.nbr;
    DBuf<int> T2(n2), P2(n2);
    k_row_info<<<blocks_for((int64_t)n2 * 32, 256, kSMs * 8), 256, 0, s>>>(A, B, C.rp.p, rows2, n2, T2.p, P2.p);
    FS_LAUNCHED();
    std::vector<int> hr(n2), ht(n2), hp(n2);
    FS_CUDA(cudaMemcpyAsync(hr.data(), rows2, sizeof(int) * n2, cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaMemcpyAsync(ht.data(), T2.p, sizeof(int) * n2, cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaMemcpyAsync(hp.data(), P2.p, sizeof(int) * n2, cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    // the task size: kTaskT products, doubled until the partial sums fit the scratch bound
    int64_t chunk = task_min;
    for (;;) {
      size_t bytes = 0;
      for (int w = 0; w < n2; w++) {
        const int64_t nt = std::max<int64_t>(1, (ht[w] + chunk - 1) / chunk);
        if (nt > 1) bytes += (size_t)nt * hp[w] * BS * sizeof(T);
      }
      if (bytes <= kSplitScratch) break;
      chunk *= 2;
    }
    std::vector<SpgemmTask> tasks;
    std::vector<SplitRow> split;
    int64_t soff = 0;
    for (int w = 0; w < n2; w++) {
      const int np = ht[w];
      const int nt = (int)std::max<int64_t>(1, (np + chunk - 1) / chunk);
      if (nt == 1) {
        tasks.push_back({hr[w], 0, np, -1});
        continue;
      }
      for (int k = 0; k < nt; k++)
        tasks.push_back({hr[w], (int)((int64_t)np * k / nt), (int)((int64_t)np * (k + 1) / nt),
                         soff + (int64_t)k * hp[w] * BS});
      split.push_back({hr[w], nt, hp[w], soff});
      soff += (int64_t)nt * hp[w] * BS;
    }
    nsplit = (int)split.size();
    dtasks.alloc(tasks.size());
    ntask.alloc(1);
    const int nt_all = (int)tasks.size();
    FS_CUDA(cudaMemcpyAsync(dtasks.p, tasks.data(), sizeof(SpgemmTask) * tasks.size(), cudaMemcpyHostToDevice, s));
    FS_CUDA(cudaMemcpyAsync(ntask.p, &nt_all, sizeof(int), cudaMemcpyHostToDevice, s));
    if (nsplit) {
      dsplit.alloc(nsplit);
      scratch.alloc((size_t)soff);
      FS_CUDA(cudaMemcpyAsync(dsplit.p, split.data(), sizeof(SplitRow) * nsplit, cudaMemcpyHostToDevice, s));
    }
    launch_mp<T, BR, BK, BC, true>(A, B, C, nullptr, ntask.p, dtasks.p, scratch.p, rc.caps[2], rc.capa[2], kSegT,
                                flags.p, s);
    if (nsplit) {
      k_sum_split<<<blocks_for((int64_t)nsplit * 32, 256, kSMs * 8), 256, 0, s>>>(dsplit.p, nsplit, C.rp.p,
                                                                                  scratch.p, BS, C.val.p);
      FS_LAUNCHED();
    }
    // the host vectors above go out of scope only after the copies that read them
    FS_CUDA(cudaStreamSynchronize(s));
  }
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
  const size_t per_slot = BS * sizeof(T) + sizeof(int);
  const size_t fixed = (size_t)4 * kProdChunk * BR * sizeof(int);
  const int ctiers[3] = {64, 256, kListCap};
  FS_REQUIRE(umax <= kListCap, FC_INTERNAL, "spgemm: product row longer than the symbolic pass allows");
  int ulo = 0;
  for (int t = 0; t < 3 && ulo < umax; t++) {
    const int ucap = ctiers[t];
    int wpb = 8;
    while (wpb > 1 && (size_t)wpb * (ucap * per_slot + fixed) > 200 * 1024) wpb >>= 1;
    const size_t shm = (size_t)wpb * (ucap * per_slot + fixed);
    auto kern = k_spgemm_numeric_sh<T, BR, BK, BC>;
    FS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    kern<<<kSMs * 8, wpb * 32, shm, s>>>(A, B, C.rp.p, C.ci.p, C.val.p, pending.p, ulo, ucap);
    FS_LAUNCHED();
    ulo = ucap;
  }
}

}  // namespace

namespace {
template <typename T>
void numeric_any(const BsrView<T> &A, const BsrView<T> &B, Bsr<T> &C, cudaStream_t s) {
  const int sh = A.br * 100 + A.bc * 10 + B.bc;
  switch (sh) {
    case 333: numeric<T, 3, 3, 3>(A, B, C, s); break;
    case 313: numeric<T, 3, 1, 3>(A, B, C, s); break;
    case 111: numeric<T, 1, 1, 1>(A, B, C, s); break;
    case 331: numeric<T, 3, 3, 1>(A, B, C, s); break;
    case 133: numeric<T, 1, 3, 3>(A, B, C, s); break;
    default: throw Error(FC_BAD_ARG, "spgemm: unsupported block shapes");
  }
}
}  // namespace

template <typename T>
void spgemm_numeric(const BsrView<T> &A, const BsrView<T> &B, Bsr<T> &C, cudaStream_t s) {
  FS_REQUIRE(A.bc == B.br && A.nbc == B.nbr && C.nbr == A.nbr && C.nbc == B.nbc && C.br == A.br && C.bc == B.bc,
             FC_BAD_ARG, "spgemm_numeric: shape mismatch");
  if (C.nnzb == 0) return;
  numeric_any<T>(A, B, C, s);
}
template void spgemm_numeric<double>(const BsrView<double> &, const BsrView<double> &, Bsr<double> &, cudaStream_t);
template void spgemm_numeric<float>(const BsrView<float> &, const BsrView<float> &, Bsr<float> &, cudaStream_t);

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

namespace {
// the sparsity pattern only (the symbolic kernel reads no values)
template <typename T>
BsrView<double> pattern_view(const BsrView<T> &M) {
  BsrView<double> v;
  v.nbr = M.nbr; v.nbc = M.nbc; v.br = M.br; v.bc = M.bc; v.nnzb = M.nnzb;
  v.rp = M.rp; v.ci = M.ci; v.val = nullptr;
  return v;
}
}  // namespace

template <typename T>
Bsr<T> spgemm(const BsrView<T> &At, const BsrView<T> &Bt, cudaStream_t s) {
  FS_REQUIRE(At.bc == Bt.br && At.nbc == Bt.nbr, FC_BAD_ARG, "spgemm: shape mismatch");
  const BsrView<double> A = pattern_view(At), B = pattern_view(Bt);
  Bsr<T> C;
  C.shape(A.nbr, B.nbc, A.br, B.bc);
  C.rp.alloc(A.nbr + 1);
  DBuf<int> cnt(A.nbr + 1), ovf(1);
  FS_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), s));
  FS_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (A.nbr + 1), s));
  const int grid = kSMs * 8;
  PhaseTimer pt(g_verbose > 1, s, "spgemm");
  // one enumeration of the products: the count pass keeps each row's unique
  // columns in a stash sized by the row's product count (at most kListCap),
  // and the fill sorts them; rows are enumerated and hashed once instead of
  // twice.  A stash beyond kStashMax entries falls back to a second pass.
  DBuf<int> scap(A.nbr + 1), soff(A.nbr + 1), stash;
  int64_t stash_n = 0;
  if (A.nbr > 0) {
    k_stash_cap<<<blocks_for((int64_t)A.nbr * 32, 256, kSMs * 8), 256, 0, s>>>(A, B, scap.p);
    FS_LAUNCHED();
    stash_n = exclusive_scan(scap.p, soff.p, A.nbr, s);
  }
  const bool stashed = stash_n > 0 && stash_n <= kStashMax;
  if (stashed) stash.alloc((size_t)stash_n);
  if (A.nbr > 0) {
    k_spgemm_symbolic<<<grid, kWarpsPerBlock * 32, 0, s>>>(A, B, 0, cnt.p, nullptr, nullptr, ovf.p,
                                                          stashed ? stash.p : nullptr, soff.p);
    FS_LAUNCHED();
  }
  pt.mark("symbolic count");
  int64_t nnz = exclusive_scan(cnt.p, C.rp.p, A.nbr, s);
  int hovf = 0;
  FS_CUDA(cudaMemcpyAsync(&hovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!hovf, FC_INTERNAL, "spgemm: a product row has more than 768 block columns");
  C.nnzb = nnz;
  C.ci.alloc(nnz);
  C.val.alloc(nnz * C.br * C.bc);
  if (nnz == 0) return C;
  pt.mark("scan + alloc");
  if (stashed) {
    k_stash_sort<<<blocks_for((int64_t)A.nbr * 32, 256, kSMs * 16), 256, 0, s>>>(A.nbr, stash.p, soff.p, C.rp.p,
                                                                                C.ci.p);
    FS_LAUNCHED();
  } else {
    k_spgemm_symbolic<<<grid, kWarpsPerBlock * 32, 0, s>>>(A, B, 1, nullptr, C.rp.p, C.ci.p, ovf.p);
    FS_LAUNCHED();
  }
  pt.mark("symbolic fill");
  numeric_any<T>(At, Bt, C, s);
  pt.mark("numeric");
  if (g_verbose > 1)
    fprintf(stderr, "[fracsolve] spgemm %d x %d blocks (%dx%d * %dx%d): A %lld, B %lld, C %lld blocks\n", A.nbr, B.nbc,
            A.br, A.bc, B.br, B.bc, (long long)A.nnzb, (long long)B.nnzb, (long long)nnz);
  FS_CUDA(cudaStreamSynchronize(s));
  return C;
}
template Bsr<double> spgemm<double>(const BsrView<double> &, const BsrView<double> &, cudaStream_t);
template Bsr<float> spgemm<float>(const BsrView<float> &, const BsrView<float> &, cudaStream_t);

// ============================================================ sparse add
namespace {
// number of sorted columns ci[lo..hi) below c, and whether c is among them
__device__ inline int rank_below(const int *ci, int lo, int hi, int c, bool &found) {
  int a = lo, b = hi;
  while (a < b) {
    const int m = (a + b) >> 1;
    if (ci[m] < c) a = m + 1;
    else b = m;
  }
  found = a < hi && ci[a] == c;
  return a - lo;
}

// C = alpha A + beta B on the union pattern, one warp per block row.  With
// m(k) = the entries of B before entry k whose column A lacks, entry t of
// A's row lands at t + m(rank of its column in B's row), and an entry k of B
// whose column A lacks at (rank of its column in A's row) + m(k).  A row of
// B that is empty (most rows: B is the fracture coupling) is a straight copy;
// rows of B longer than kAddB entries are merged by one lane.  Each value is
// (0 + alpha a) + beta b, with absent terms skipped.
constexpr int kAddB = 64;

__global__ void __launch_bounds__(256)
    k_spadd(BsrView<double> A, BsrView<double> B, double alpha, double beta, int pass, int *cnt,
            const int *rpC, int *ciC, double *valC) {
  __shared__ int s_m[8][kAddB + 1];
  const int bs = A.br * A.bc;
  const int lane = threadIdx.x & 31;
  int *m = s_m[threadIdx.x >> 5];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < A.nbr; i += nw) {
    const int a0 = A.rp[i], na = A.rp[i + 1] - a0, b0 = B.rp[i], nb = B.rp[i + 1] - b0;
    const int o = pass ? rpC[i] : 0;
    if (nb == 0) {
      if (!pass) {
        if (lane == 0) cnt[i] = na;
        continue;
      }
      for (int t = lane; t < na; t += 32) ciC[o + t] = A.ci[a0 + t];
      for (int64_t q = lane; q < (int64_t)na * bs; q += 32)
        valC[(int64_t)o * bs + q] = 0.0 + alpha * A.val[(int64_t)a0 * bs + q];
      continue;
    }
    if (nb > kAddB) {   // long rows of B: a sequential merge
      if (lane == 0) {
        int a = a0, ae = a0 + na, b = b0, be = b0 + nb, n = 0;
        while (a < ae || b < be) {
          const int ca = a < ae ? A.ci[a] : INT32_MAX, cb = b < be ? B.ci[b] : INT32_MAX;
          const int c = ca < cb ? ca : cb;
          if (pass) {
            ciC[o + n] = c;
            for (int q = 0; q < bs; q++) {
              double v = 0.0;
              if (ca == c) v += alpha * A.val[(int64_t)a * bs + q];
              if (cb == c) v += beta * B.val[(int64_t)b * bs + q];
              valC[(int64_t)(o + n) * bs + q] = v;
            }
          }
          if (ca == c) a++;
          if (cb == c) b++;
          n++;
        }
        if (!pass) cnt[i] = n;
      }
      __syncwarp();
      continue;
    }
    // m: exclusive prefix over B's row of "column absent from A"
    int carry = 0;
    for (int k0 = 0; k0 < nb; k0 += 32) {
      const int k = k0 + lane;
      int absent = 0;
      if (k < nb) {
        bool f;
        rank_below(A.ci, a0, a0 + na, B.ci[b0 + k], f);
        absent = !f;
      }
      int inc = absent;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
      }
      if (k < nb) m[k] = carry + inc - absent;
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) m[nb] = carry;
    __syncwarp();
    if (!pass) {
      if (lane == 0) cnt[i] = na + m[nb];
      __syncwarp();
      continue;
    }
    for (int t = lane; t < na; t += 32) {
      const int c = A.ci[a0 + t];
      bool f;
      const int r = rank_below(B.ci, b0, b0 + nb, c, f);
      const int pos = o + t + m[r];
      ciC[pos] = c;
      for (int q = 0; q < bs; q++) {
        double v = 0.0;
        v += alpha * A.val[(int64_t)(a0 + t) * bs + q];
        if (f) v += beta * B.val[(int64_t)(b0 + r) * bs + q];
        valC[(int64_t)pos * bs + q] = v;
      }
    }
    for (int k = lane; k < nb; k += 32) {
      const int c = B.ci[b0 + k];
      bool f;
      const int r = rank_below(A.ci, a0, a0 + na, c, f);
      if (f) continue;
      const int pos = o + r + m[k];
      ciC[pos] = c;
      for (int q = 0; q < bs; q++) {
        double v = 0.0;
        v += beta * B.val[(int64_t)(b0 + k) * bs + q];
        valC[(int64_t)pos * bs + q] = v;
      }
    }
    __syncwarp();
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
  const int grid = blocks_for((int64_t)A.nbr * 32, 256, kSMs * 16);
  if (A.nbr > 0) {
    k_spadd<<<grid, 256, 0, s>>>(A, B, alpha, beta, 0, cnt.p, nullptr, nullptr, nullptr);
    FS_LAUNCHED();
  }
  int64_t nnz = exclusive_scan(cnt.p, C.rp.p, A.nbr, s);
  C.nnzb = nnz;
  C.ci.alloc(nnz);
  C.val.alloc(nnz * C.br * C.bc);
  if (nnz) {
    k_spadd<<<grid, 256, 0, s>>>(A, B, alpha, beta, 1, nullptr, C.rp.p, C.ci.p, C.val.p);
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
template Bsr<double> copy_cast<double, float>(const BsrView<float> &, cudaStream_t);
template Bsr<float> copy_cast<float, float>(const BsrView<float> &, cudaStream_t);

// ============================================================ sliced ELL
namespace {
template <typename TI>
__global__ void k_sell_width(BsrView<TI> A, int nslice, int *w) {
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

// Lane order of a jagged slice: the row at position r of slice sl goes to
// lane = (number of the slice's rows that are longer) + (number of equally
// long rows before it); rows past the matrix count as empty and come last.
template <typename TI>
__global__ void k_sell_sort(BsrView<TI> A, int nslice, int *lm) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nslice * kSellH;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = t / kSellH;
    const int r = (int)(t % kSellH);
    const int len = t < A.nbr ? A.rp[t + 1] - A.rp[t] : 0;
    int lane = 0;
    for (int q = 0; q < kSellH; q++) {
      const int64_t u = sl * kSellH + q;
      const int lq = u < A.nbr ? A.rp[u + 1] - A.rp[u] : 0;
      lane += lq > len || (lq == len && q < r);
    }
    lm[sl * kSellH + lane] = (len << 5) | r;
  }
}

// a jagged slice starts at the row pointer of its first row
template <typename TI>
__global__ void k_jag_offsets(BsrView<TI> A, int nslice, int64_t *sp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nslice;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i * kSellH < A.nbr ? i * kSellH : A.nbr;
    sp[i] = A.rp[r];
  }
}

template <typename T, typename TI>
__global__ void k_sell_fill(BsrView<TI> A, int nslice, const int64_t *sp, int *ci, T *val) {
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

// jagged fill: one warp per slice, the same slot walk as the product kernel
template <typename T, typename TI>
__global__ void k_sell_fill_jag(BsrView<TI> A, int nslice, const int64_t *sp, const int *lm, int *ci, T *val) {
  const int bs = A.br * A.bc;
  const int lane = (int)(threadIdx.x % kSellH);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) / kSellH;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kSellH; sl < nslice; sl += nwarp) {
    const int m = lm[sl * kSellH + lane];
    const int len = m >> 5;
    const int64_t row = sl * kSellH + (m & 31);
    const int b0 = row < A.nbr ? A.rp[row] : 0;
    const int w = __shfl_sync(0xffffffffu, len, 0);
    int64_t off = sp[sl];
    for (int k = 0; k < w; k++) {
      const int ak = __popc(__ballot_sync(0xffffffffu, k < len));
      if (k < len) {
        ci[off + lane] = A.ci[b0 + k];
        for (int q = 0; q < bs; q++) val[(off * bs) + (int64_t)q * ak + lane] = (T)A.val[(int64_t)(b0 + k) * bs + q];
      }
      off += ak;
    }
  }
}
}  // namespace

template <typename T, typename TI>
Sell<T> to_sell(const BsrView<TI> &A, cudaStream_t s) {
  Sell<T> S;
  S.nbr = A.nbr; S.nbc = A.nbc; S.br = A.br; S.bc = A.bc; S.nnzb = A.nnzb;
  S.nslice = (A.nbr + kSellH - 1) / kSellH;
  S.sp.alloc(S.nslice + 1);
  if (S.nslice == 0) {
    FS_CUDA(cudaMemsetAsync(S.sp.p, 0, sizeof(int64_t), s));
    return S;
  }
  const int bs = A.br * A.bc;
  DBuf<int> w(S.nslice + 1), wp(S.nslice + 1);
  k_sell_width<TI><<<blocks_for(S.nslice, 128, kSMs * 8), 128, 0, s>>>(A, S.nslice, w.p);
  FS_LAUNCHED();
  const int64_t slots = exclusive_scan(w.p, wp.p, S.nslice, s);
  const double padded = (double)slots * kSellH;
  // every slice is at most `slots` wide, so the row lengths fit the 27 bits
  // of a lane entry
  bool jag = padded > kSellJagPadding * (double)A.nnzb &&
             padded * (bs * sizeof(T) + sizeof(int)) > kSellJagMinBytes && slots < (int64_t(1) << 26);
  // test hook, compiled only into the test build (FS_TEST_HOOKS):
  // FS_SELL_FORCE_JAG=1 makes every sliced-ELL copy jagged, so that small
  // problems run the layout only large ones choose
#ifdef FS_TEST_HOOKS
  if (const char *ev = std::getenv("FS_SELL_FORCE_JAG"))
    if (std::strtol(ev, nullptr, 10) == 1 && slots < (int64_t(1) << 26)) jag = true;
#endif
  if (jag) {
    S.lm.alloc((size_t)S.nslice * kSellH);
    k_sell_sort<TI><<<blocks_for((int64_t)S.nslice * kSellH, 128, kSMs * 16), 128, 0, s>>>(A, S.nslice, S.lm.p);
    FS_LAUNCHED();
    k_jag_offsets<TI><<<blocks_for(S.nslice + 1, 256, kSMs * 4), 256, 0, s>>>(A, S.nslice, S.sp.p);
    FS_LAUNCHED();
    S.ci.alloc((size_t)A.nnzb + kSellH);
    S.val.alloc(((size_t)A.nnzb + kSellH) * bs);
    if (A.nnzb) {
      k_sell_fill_jag<T, TI><<<blocks_for((int64_t)S.nslice * kSellH, 128, kSMs * 16), 128, 0, s>>>(
          A, S.nslice, S.sp.p, S.lm.p, S.ci.p, S.val.p);
      FS_LAUNCHED();
    }
    return S;
  }
  k_to_i64<<<blocks_for(S.nslice + 1, 256, kSMs * 4), 256, 0, s>>>(wp.p, S.sp.p, S.nslice);
  FS_LAUNCHED();
  S.ci.alloc(slots * kSellH);
  S.val.alloc(slots * kSellH * bs);
  if (slots) {
    k_sell_fill<T, TI><<<blocks_for((int64_t)S.nslice * kSellH, 128, kSMs * 16), 128, 0, s>>>(A, S.nslice, S.sp.p,
                                                                                          S.ci.p, S.val.p);
    FS_LAUNCHED();
  }
  return S;
}
namespace {
// a slice of rows [r0, r0 + 32 / g) starts after all entries of the rows before
template <typename TQ>
__global__ void k_jag_offsets(BsrView<double> P, BsrView<TQ> Q, bool two, int rps, int nslice, int64_t *sp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nslice;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i * rps < P.nbr ? i * rps : P.nbr;
    sp[i] = (int64_t)P.rp[r] + (two ? Q.rp[r] : 0);
  }
}

// one warp per slice, the slot walk of k_jag_spmv
template <typename T, typename TQ>
__global__ void k_jag_fill(BsrView<double> P, BsrView<TQ> Q, bool two, int g, int nslice, const int64_t *sp,
                           int2 *len, int *ci, T *val) {
  const int bs = P.br * P.bc;
  const int lane = (int)(threadIdx.x % kSellH);
  const int j = lane % g, rps = kSellH / g;
  const unsigned below = (1u << lane) - 1u;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) / kSellH;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kSellH; sl < nslice; sl += nwarp) {
    const int64_t row = sl * rps + lane / g;
    const bool real = row < P.nbr;
    const int p0 = real ? P.rp[row] : 0, lp = real ? P.rp[row + 1] - p0 : 0;
    const int q0 = real && two ? Q.rp[row] : 0, lq = real && two ? Q.rp[row + 1] - q0 : 0;
    const int L = lp + lq;
    if (real && j == 0) len[row] = make_int2(lp, L);
    int w = (L + g - 1) / g;
    for (int o = kSellH / 2; o; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    int64_t off = sp[sl];
    for (int k = 0; k < w; k++) {
      const int e = j + g * k;
      const bool on = e < L;
      const unsigned act = __ballot_sync(0xffffffffu, on);
      const int ak = __popc(act);
      if (on) {
        const int rk = __popc(act & below);
        T *v = val + off * bs + rk;
        if (e < lp) {
          ci[off + rk] = P.ci[p0 + e];
          for (int q = 0; q < bs; q++) v[(int64_t)q * ak] = (T)P.val[(int64_t)(p0 + e) * bs + q];
        } else {
          const int ee = e - lp;
          ci[off + rk] = Q.ci[q0 + ee];
          for (int q = 0; q < bs; q++) v[(int64_t)q * ak] = (T)Q.val[(int64_t)(q0 + ee) * bs + q];
        }
      }
      off += ak;
    }
  }
}
}  // namespace

template <typename T, typename TQ>
Jag<T> to_jag(const BsrView<double> &P, const BsrView<TQ> *Q, int g, cudaStream_t s) {
  FS_REQUIRE(g == 1 || g == 4 || g == 8 || g == 16 || g == 32, FC_INTERNAL, "to_jag: lanes per row");
  FS_REQUIRE(!Q || (P.nbr == Q->nbr && P.nbc == Q->nbc && P.br == Q->br && P.bc == Q->bc), FC_INTERNAL,
             "to_jag: the two matrices differ in shape");
  const BsrView<TQ> q = Q ? *Q : BsrView<TQ>();
  Jag<T> J;
  J.nbr = P.nbr; J.nbc = P.nbc; J.br = P.br; J.bc = P.bc; J.g = g;
  J.nnzb = P.nnzb + (Q ? Q->nnzb : 0);
  const int rps = kSellH / g;
  J.nslice = (P.nbr + rps - 1) / rps;
  J.sp.alloc((size_t)J.nslice + 1);
  J.len.alloc((size_t)std::max(P.nbr, 1));
  J.ci.alloc((size_t)J.nnzb + kSellH);
  J.val.alloc(((size_t)J.nnzb + kSellH) * P.br * P.bc);
  k_jag_offsets<TQ><<<blocks_for(J.nslice + 1, 256, kSMs * 4), 256, 0, s>>>(P, q, Q != nullptr, rps, J.nslice,
                                                                            J.sp.p);
  FS_LAUNCHED();
  if (J.nslice) {
    k_jag_fill<T, TQ><<<blocks_for((int64_t)J.nslice * kSellH, 128, kSMs * 16), 128, 0, s>>>(
        P, q, Q != nullptr, g, J.nslice, J.sp.p, J.len.p, J.ci.p, J.val.p);
    FS_LAUNCHED();
  }
  return J;
}
template Jag<float> to_jag<float, float>(const BsrView<double> &, const BsrView<float> *, int, cudaStream_t);
template Jag<double> to_jag<double, double>(const BsrView<double> &, const BsrView<double> *, int, cudaStream_t);

namespace {
__global__ void k_chunk_count(BsrView<double> A, int g, int *cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.nbr; r += (int64_t)gridDim.x * blockDim.x)
    cnt[r] = (A.rp[r + 1] - A.rp[r] + g - 1) / g;
}

// one warp per row: position p of the row's padded chunks is entry p of the
// row (chunk p / g, lane p % g)
template <typename T>
__global__ void k_chunk_fill(BsrView<double> A, int g, const int *rc, int *ci, T *val) {
  const int bs = A.br * A.bc;
  const int lane = (int)(threadIdx.x & 31);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < A.nbr; r += nwarp) {
    const int b0 = A.rp[r], len = A.rp[r + 1] - b0;
    const int64_t c0 = rc[r];
    const int npos = (rc[r + 1] - rc[r]) * g;
    for (int p = lane; p < npos; p += 32) {
      const int64_t c = c0 + p / g;
      const int j = p % g;
      const bool real = p < len;
      ci[c * g + j] = real ? A.ci[b0 + p] : 0;
      for (int q = 0; q < bs; q++)
        val[(c * bs + q) * g + j] = real ? (T)A.val[(int64_t)(b0 + p) * bs + q] : T(0);
    }
  }
}
}  // namespace

template <typename T>
Chunked<T> to_chunked(const BsrView<double> &A, int g, cudaStream_t s) {
  FS_REQUIRE(g == 4 || g == 8 || g == 16 || g == 32, FC_INTERNAL, "to_chunked: lanes per row");
  Chunked<T> C;
  C.nbr = A.nbr; C.nbc = A.nbc; C.br = A.br; C.bc = A.bc; C.g = g; C.nnzb = A.nnzb;
  C.rc.alloc((size_t)A.nbr + 1);
  if (A.nbr == 0) {
    FS_CUDA(cudaMemsetAsync(C.rc.p, 0, sizeof(int), s));
    return C;
  }
  DBuf<int> cnt((size_t)A.nbr + 1);
  k_chunk_count<<<blocks_for(A.nbr, 256, kSMs * 8), 256, 0, s>>>(A, g, cnt.p);
  FS_LAUNCHED();
  C.nchunk = exclusive_scan(cnt.p, C.rc.p, A.nbr, s);
  C.ci.alloc((size_t)std::max<int64_t>(C.nchunk, 1) * g);
  C.val.alloc((size_t)std::max<int64_t>(C.nchunk, 1) * A.br * A.bc * g);
  if (C.nchunk) {
    k_chunk_fill<T><<<blocks_for((int64_t)A.nbr * 32, 256, kSMs * 16), 256, 0, s>>>(A, g, C.rc.p, C.ci.p, C.val.p);
    FS_LAUNCHED();
  }
  return C;
}
template Chunked<float> to_chunked<float>(const BsrView<double> &, int, cudaStream_t);
template Chunked<double> to_chunked<double>(const BsrView<double> &, int, cudaStream_t);

template Sell<float> to_sell<float, double>(const BsrView<double> &, cudaStream_t);
template Sell<double> to_sell<double, double>(const BsrView<double> &, cudaStream_t);
template Sell<float> to_sell<float, float>(const BsrView<float> &, cudaStream_t);

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
