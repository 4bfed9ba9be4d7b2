// Block sparse matrix-vector products with fused epilogues.
//
// BSR kernel: one group of G lanes owns one block row; each lane takes whole
// blocks of the row (its values, column and the BC entries of x it needs),
// the group reduces the BR partial sums with shuffles, and lane 0 hands them
// to an epilogue that finishes the row (axpby, Chebyshev update, H~^-1
// solve).  Used for long rows (restriction) and setup products; the short-row
// products of the solve use the sliced-ELL kernel of sell.cuh.
#pragma once

#include "common.cuh"

namespace fs {

template <int G, typename T>
__device__ inline T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

template <int BR, int BC, int G, typename TA, typename TX, typename Epi>
__global__ void __launch_bounds__(256) k_bsr_spmv(BsrView<TA> A, const TX *__restrict__ x, Epi epi) {
  constexpr int BS = BR * BC;
  const int lane = threadIdx.x & (G - 1);
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const bool valid = row < A.nbr;
  TA acc[BR];
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = TA(0);
  if (valid) {
    const int s = __ldg(A.rp + row), e = __ldg(A.rp + row + 1);
    // each lane takes whole blocks: no index arithmetic per scalar entry
#pragma unroll 4
    for (int b = s + lane; b < e; b += G) {
      const int col = __ldg(A.ci + b);
      TA a[BS];
#pragma unroll
      for (int q = 0; q < BS; q++) a[q] = __ldg(A.val + (int64_t)b * BS + q);
      TA xv[BC];
#pragma unroll
      for (int j = 0; j < BC; j++) xv[j] = (TA)__ldg(x + (int64_t)col * BC + j);
#pragma unroll
      for (int r = 0; r < BR; r++)
#pragma unroll
        for (int j = 0; j < BC; j++) acc[r] += a[r * BC + j] * xv[j];
    }
  }
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = group_sum<G>(acc[q]);
  if (valid && lane == 0) epi(row, acc);
}

// y[row] = alpha * (A x)[row] + beta * z[row]   (z may alias y; z unused if beta == 0)
template <int BR, typename TA, typename TY, typename TZ>
struct EpiAxpby {
  TY *y;
  const TZ *z;
  TA alpha, beta;
  __device__ void operator()(int64_t row, const TA *acc) const {
#pragma unroll
    for (int q = 0; q < BR; q++) {
      TA v = alpha * acc[q];
      if (beta != TA(0)) v += beta * (TA)z[row * BR + q];
      y[row * BR + q] = (TY)v;
    }
  }
};

// y[row] = Dinv[row] * (A x)[row]   (power iteration on D^-1 S)
template <int BR, typename TA>
struct EpiBlockDiag {
  TA *y;
  const TA *Dinv;
  __device__ void operator()(int64_t row, const TA *acc) const {
    const TA *D = Dinv + row * BR * BR;
#pragma unroll
    for (int a = 0; a < BR; a++) {
      TA s = 0;
#pragma unroll
      for (int b = 0; b < BR; b++) s += D[a * BR + b] * acc[b];
      y[row * BR + a] = s;
    }
  }
};

// Chebyshev step (Saad, Alg. 12.1) fused with the residual:
//   r = f - (S x_in)[row];  d = cd * d + cr * Dinv r;  x_out = x_in + d
template <int BR, typename TA>
struct EpiCheb {
  const TA *f;
  const TA *x_in;
  TA *x_out;
  TA *d;
  const TA *Dinv;
  TA cd, cr;
  __device__ void operator()(int64_t row, const TA *acc) const {
    TA r[BR];
#pragma unroll
    for (int q = 0; q < BR; q++) r[q] = f[row * BR + q] - acc[q];
    const TA *D = Dinv + row * BR * BR;
#pragma unroll
    for (int a = 0; a < BR; a++) {
      TA s = 0;
#pragma unroll
      for (int b = 0; b < BR; b++) s += D[a * BR + b] * r[b];
      TA dn = cr * s;
      if (cd != TA(0)) dn += cd * d[row * BR + a];
      d[row * BR + a] = dn;
      x_out[row * BR + a] = x_in[row * BR + a] + dn;
    }
  }
};

// The prolongation of a V-cycle level fused with the first post-smoothing
// step (a Chebyshev step from the corrected iterate, no previous direction).
// With x1 = x + P x_c, the residual f - S x1 equals r - (S P) x_c, where
// r = f - S x is the residual already formed for the restriction, so the step
// reads P and S P instead of P and S:
//   x1 = x + acc1;  d = cr Dinv (r - acc2);  x_out = x1 + d
// (acc1 = (P x_c)[row], acc2 = (S P x_c)[row]).
template <int BR, typename TA>
struct EpiProlongCheb {
  const TA *x;
  const TA *r;
  const TA *Dinv;
  TA *x_out;
  TA *d;
  TA cr;
  __device__ void operator()(int64_t row, const TA *acc1, const TA *acc2) const {
    TA res[BR];
#pragma unroll
    for (int q = 0; q < BR; q++) res[q] = r[row * BR + q] - acc2[q];
    const TA *D = Dinv + row * BR * BR;
#pragma unroll
    for (int a = 0; a < BR; a++) {
      TA s = 0;
#pragma unroll
      for (int b = 0; b < BR; b++) s += D[a * BR + b] * res[b];
      const TA dn = cr * s;
      d[row * BR + a] = dn;
      const TA x1 = x[row * BR + a] + acc1[a];
      x_out[row * BR + a] = x1 + dn;
    }
  }
};

// The last step of Alg. 2 and Alg. 4 fused with the C2 product:
//   v_t[row] = -t_t[row] + Hinv[row] * (C2 v_u)[row]
template <typename TA>
struct EpiHinvUpdate {
  TA *v_t;
  const TA *t_t;
  const TA *Hinv;
  __device__ void operator()(int64_t row, const TA *acc) const {
    const TA *Hi = Hinv + row * 9;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      TA s = 0;
#pragma unroll
      for (int b = 0; b < 3; b++) s += Hi[a * 3 + b] * acc[b];
      v_t[row * 3 + a] = -t_t[row * 3 + a] + s;
    }
  }
};

// One block of 256 threads per row, for matrices with few, very long rows
// (the restrictions of the coarse levels: ~100-5000 rows of hundreds of
// blocks): each thread takes whole blocks with a stride of 256, the warps
// reduce with shuffles and the block through shared memory, and thread 0
// hands the sums to the epilogue.
template <int BR, int BC, typename TA, typename TX, typename Epi>
__global__ void __launch_bounds__(256) k_bsr_spmv_rowcta(BsrView<TA> A, const TX *__restrict__ x, Epi epi) {
  constexpr int BS = BR * BC;
  __shared__ TA part[8][BR];
  const int64_t row = blockIdx.x;
  const int s = __ldg(A.rp + row), e = __ldg(A.rp + row + 1);
  TA acc[BR];
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = TA(0);
  for (int b = s + threadIdx.x; b < e; b += 256) {
    const int col = __ldg(A.ci + b);
    TA xv[BC];
#pragma unroll
    for (int j = 0; j < BC; j++) xv[j] = (TA)__ldg(x + (int64_t)col * BC + j);
#pragma unroll
    for (int r = 0; r < BR; r++)
#pragma unroll
      for (int j = 0; j < BC; j++) acc[r] += __ldg(A.val + (int64_t)b * BS + r * BC + j) * xv[j];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < BR; q++) {
    const TA v = group_sum<32>(acc[q]);
    if (lane == 0) part[wid][q] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < BR; q++) {
      TA v = part[0][q];
      for (int w = 1; w < 8; w++) v += part[w][q];
      acc[q] = v;
    }
    epi(row, acc);
  }
}

// rows of at least this many blocks on average, in a matrix of at most
// kRowCtaMaxRows rows, take one block of threads each
constexpr double kRowCtaMinMean = 200.0;
constexpr int kRowCtaMaxRows = 8 * 152 * 4;
// a matrix with few, very long rows (coarse restrictions) goes to the
// one-block-per-row kernel
inline bool rowcta_rows(int64_t nnzb, int nbr) {
  return nbr > 0 && nbr <= kRowCtaMaxRows && (double)nnzb / nbr >= kRowCtaMinMean;
}

// lanes per row from the mean number of blocks per row (sweeps on the
// 128^3 workload, coarse part of the cycle: for the ~69-block rows of the
// first coarse level 8 lanes 0.359 ms, 16 lanes 0.373 ms, 32 lanes
// 0.425 ms; the ~126-block rows of the finest restriction keep 32)
#ifndef FS_BSR_LANES32_ABOVE
#define FS_BSR_LANES32_ABOVE 100.0
#endif
#ifndef FS_BSR_LANES16_ABOVE
#define FS_BSR_LANES16_ABOVE 100.0
#endif
inline int lanes_for(int64_t nnzb, int nbr, int bs) {
  (void)bs;
  double per = nbr > 0 ? (double)nnzb / nbr : 0.0;
  if (per > FS_BSR_LANES32_ABOVE) return 32;
  if (per > FS_BSR_LANES16_ABOVE) return 16;
  if (per > 6) return 8;
  return 4;
}

template <int BR, int BC, int G, typename TA, typename TX, typename Epi>
inline void spmv_g(const BsrView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  const int threads = 256;
  const int64_t nthreads = (int64_t)A.nbr * G;
  const int64_t blocks = (nthreads + threads - 1) / threads;
  k_bsr_spmv<BR, BC, G, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi);
  FS_LAUNCHED();
}

// Launch with a lane count chosen from the mean scalar entries per row.
template <int BR, int BC, typename TA, typename TX, typename Epi>
inline void spmv(const BsrView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  if (A.nbr <= 0) return;
  if (rowcta_rows(A.nnzb, A.nbr)) {
    k_bsr_spmv_rowcta<BR, BC, TA, TX, Epi><<<(unsigned)A.nbr, 256, 0, s>>>(A, x, epi);
    FS_LAUNCHED();
    return;
  }
  switch (lanes_for(A.nnzb, A.nbr, BR * BC)) {
    case 32: spmv_g<BR, BC, 32>(A, x, epi, s); break;
    case 16: spmv_g<BR, BC, 16>(A, x, epi, s); break;
    case 8: spmv_g<BR, BC, 8>(A, x, epi, s); break;
    default: spmv_g<BR, BC, 4>(A, x, epi, s); break;
  }
}

// Chunked BSR for long rows: a row's blocks in chunks of G (the lanes of
// its group), each chunk stored slot-major and 32-byte aligned: G column
// indices, then each of the BR*BC block scalars as G consecutive values; the
// last chunk of a row is padded with zero blocks of column 0.  Lane j of a
// group takes entry j of every chunk of its row, so each load a group issues
// is G consecutive values (one 32-byte sector for G = 8 floats) where the BSR
// kernel's lanes read their 36-byte blocks scalar by scalar (ncu: ~20 sectors
// per load request there, the load queue the first stall).
template <typename T>
struct ChunkView {
  int nbr = 0, nbc = 0, br = 0, bc = 0, g = 8;
  int64_t nnzb = 0;                 // blocks of the matrix (without the padding)
  const int *rc = nullptr;          // nbr + 1 chunk offsets
  const int *ci = nullptr;          // chunks * g
  const T *val = nullptr;           // chunks * br * bc * g
};

template <typename T>
struct Chunked {
  int nbr = 0, nbc = 0, br = 0, bc = 0, g = 8;
  int64_t nnzb = 0, nchunk = 0;
  DBuf<int> rc, ci;
  DBuf<T> val;
  ChunkView<T> view() const {
    ChunkView<T> v;
    v.nbr = nbr; v.nbc = nbc; v.br = br; v.bc = bc; v.g = g; v.nnzb = nnzb;
    v.rc = rc.p; v.ci = ci.p; v.val = val.p;
    return v;
  }
};

#ifndef FS_CHUNK_UNROLL
#define FS_CHUNK_UNROLL 4
#endif
// chunks of a row in flight per lane (128^3 sweep, coarse part of the cycle:
// 2 / 4 / 8 gave 0.302 / 0.303 / 0.307 ms: the pass is latency-bound either way)
constexpr int kChunkUnroll = FS_CHUNK_UNROLL;

template <int BR, int BC, int G, typename TA, typename TX, typename Epi>
__global__ void __launch_bounds__(256) k_chunk_spmv(ChunkView<TA> A, const TX *__restrict__ x, Epi epi) {
  constexpr int BS = BR * BC;
  const int lane = threadIdx.x & (G - 1);
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const bool valid = row < A.nbr;
  TA acc[BR];
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = TA(0);
  if (valid) {
    const int c0 = __ldg(A.rc + row), c1 = __ldg(A.rc + row + 1);
#pragma unroll kChunkUnroll
    for (int c = c0; c < c1; c++) {
      const int col = __ldg(A.ci + (int64_t)c * G + lane);
      const TA *__restrict__ v = A.val + (int64_t)c * BS * G + lane;
      TA a[BS];
#pragma unroll
      for (int q = 0; q < BS; q++) a[q] = __ldg(v + q * G);
      TA xv[BC];
#pragma unroll
      for (int j = 0; j < BC; j++) xv[j] = (TA)__ldg(x + (int64_t)col * BC + j);
#pragma unroll
      for (int r = 0; r < BR; r++)
#pragma unroll
        for (int j = 0; j < BC; j++) acc[r] += a[r * BC + j] * xv[j];
    }
  }
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = group_sum<G>(acc[q]);
  if (valid && lane == 0) epi(row, acc);
}

template <int BR, int BC, typename TA, typename TX, typename Epi>
inline void chunk_spmv(const ChunkView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  if (A.nbr <= 0) return;
  const int threads = 256;
  const int64_t blocks = ((int64_t)A.nbr * A.g + threads - 1) / threads;
  switch (A.g) {
    case 32: k_chunk_spmv<BR, BC, 32, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    case 16: k_chunk_spmv<BR, BC, 16, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    case 8: k_chunk_spmv<BR, BC, 8, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    default: k_chunk_spmv<BR, BC, 4, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
  }
  FS_LAUNCHED();
}

// y = alpha A x + beta z
template <int BR, int BC, typename TA, typename TX, typename TY, typename TZ>
inline void spmv_axpby(const BsrView<TA> &A, const TX *x, TY *y, double alpha, double beta,
                       const TZ *z, cudaStream_t s) {
  EpiAxpby<BR, TA, TY, TZ> e{y, z, (TA)alpha, (TA)beta};
  spmv<BR, BC>(A, x, e, s);
}

}  // namespace fs
