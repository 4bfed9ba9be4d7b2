// Sliced-ELL storage of block sparse matrices for the solve-phase products.
//
// Block rows are grouped in slices of kSellH = 32 (one warp, one thread per
// block row).  A slice is padded to the longest row it holds; its entries
// are stored slot-major across its rows, so for entry slot k of a slice the
// 32 column indices are 32 consecutive ints and each of the BR*BC block
// values is 32 consecutive scalars: every load a warp issues for the matrix
// is one fully used, coalesced line.  (8-row slices cut the padding of the
// prolongator from 47% to 29% but made the finest-level smoother 9% slower:
// four 32-byte pieces per warp load instead of one line.)  Padding entries
// point at column 0 with zero values.  Each thread accumulates its own BR
// outputs in registers, so there is no cross-lane reduction and the epilogue
// runs on all lanes at once.
#pragma once

#include "common.cuh"
#include "spmv.cuh"

namespace fs {

constexpr int kSellH = 32;   // block rows per slice

template <typename T>
struct SellView {
  int nbr = 0, nbc = 0, br = 0, bc = 0, nslice = 0;
  int64_t slots = 0;           // sum over slices of their widths
  const int64_t *sp = nullptr; // nslice + 1 slot offsets
  const int *ci = nullptr;     // slots * kSellH
  const T *val = nullptr;      // slots * br * bc * kSellH
};

template <typename T>
struct Sell {
  int nbr = 0, nbc = 0, br = 0, bc = 0, nslice = 0;
  int64_t slots = 0, nnzb = 0;
  DBuf<int64_t> sp;
  DBuf<int> ci;
  DBuf<T> val;
  SellView<T> view() const {
    SellView<T> v;
    v.nbr = nbr; v.nbc = nbc; v.br = br; v.bc = bc; v.nslice = nslice; v.slots = slots;
    v.sp = sp.p; v.ci = ci.p; v.val = val.p;
    return v;
  }
};

// Convert a double BSR matrix (sorted rows) into sliced ELL of value type T.
template <typename T>
Sell<T> to_sell(const BsrView<double> &A, cudaStream_t s);

template <int BR, int BC, typename TA, typename TX, typename Epi>
__global__ void __launch_bounds__(256) k_sell_spmv(SellView<TA> A, const TX *__restrict__ x, Epi epi) {
  constexpr int BS = BR * BC;
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t slice = row / kSellH;
  const int lane = (int)(row % kSellH);
  if (slice >= A.nslice) return;
  const int64_t s0 = A.sp[slice], s1 = A.sp[slice + 1];
  TA acc[BR];
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = TA(0);
  const int *__restrict__ ci = A.ci + s0 * kSellH + lane;
  const TA *__restrict__ v = A.val + s0 * kSellH * BS + lane;
  const int w = (int)(s1 - s0);
#pragma unroll 4
  for (int k = 0; k < w; k++) {
    const int c = __ldg(ci + (int64_t)k * kSellH);
    TA a[BS];
#pragma unroll
    for (int q = 0; q < BS; q++) a[q] = __ldg(v + ((int64_t)k * BS + q) * kSellH);
    TA xv[BC];
#pragma unroll
    for (int j = 0; j < BC; j++) xv[j] = (TA)__ldg(x + (int64_t)c * BC + j);
#pragma unroll
    for (int r = 0; r < BR; r++)
#pragma unroll
      for (int j = 0; j < BC; j++) acc[r] += a[r * BC + j] * xv[j];
  }
  if (row < A.nbr) epi(row, acc);
}

template <int BR, int BC, typename TA, typename TX, typename Epi>
inline void sell_spmv(const SellView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  if (A.nbr <= 0) return;
  const int threads = 256;
  const int64_t blocks = ((int64_t)A.nslice * kSellH + threads - 1) / threads;
  k_sell_spmv<BR, BC, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi);
  FS_LAUNCHED();
}

// y = alpha A x + beta z
template <int BR, int BC, typename TA, typename TX, typename TY, typename TZ>
inline void sell_axpby(const SellView<TA> &A, const TX *x, TY *y, double alpha, double beta, const TZ *z,
                       cudaStream_t s) {
  EpiAxpby<BR, TA, TY, TZ> e{y, z, (TA)alpha, (TA)beta};
  sell_spmv<BR, BC>(A, x, e, s);
}

}  // namespace fs
