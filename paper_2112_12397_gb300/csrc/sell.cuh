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
//
// Jagged slices, for matrices with much padding (prolongators; the node rows
// of C1 and Q1, empty away from the fractures): the rows of a slice are given
// to the lanes in order of decreasing length, so at entry slot k the lanes
// that still hold an entry are a prefix of the warp, of length a_k = the
// popcount of a ballot; slot k stores only those a_k entries (a_k column
// indices, then each block scalar as a_k consecutive values), the slots of a
// slice one after the other (the jagged-diagonal layout within a slice of 32
// rows).  A slice then starts at the row pointer of its first row, and there
// is no padding to read.  The permutation stays inside the slice, so the
// epilogue's row accesses still fall in the slice's own lines.
#pragma once

#include "common.cuh"
#include "spmv.cuh"

namespace fs {

constexpr int kSellH = 32;   // block rows per slice

template <typename T>
struct SellView {
  int nbr = 0, nbc = 0, br = 0, bc = 0, nslice = 0;
  const int64_t *sp = nullptr; // nslice + 1 offsets (in slots of kSellH entries; jagged: in entries)
  const int *ci = nullptr;
  const T *val = nullptr;
  // jagged slices: nslice * kSellH lane entries (row length << 5) | position
  // of the lane's row in its slice, lanes in order of decreasing length;
  // null for padded slices (lane l holds row l)
  const int *lm = nullptr;
};

template <typename T>
struct Sell {
  int nbr = 0, nbc = 0, br = 0, bc = 0, nslice = 0;
  int64_t nnzb = 0;
  DBuf<int64_t> sp;
  DBuf<int> ci;
  DBuf<T> val;
  DBuf<int> lm;
  SellView<T> view() const {
    SellView<T> v;
    v.nbr = nbr; v.nbc = nbc; v.br = br; v.bc = bc; v.nslice = nslice;
    v.sp = sp.p; v.ci = ci.p; v.val = val.p; v.lm = lm.p;
    return v;
  }
};

// Jagged slices are used where padded slices would hold more than
// kSellJagPadding x the entries and more than kSellJagMinBytes: smaller
// operators (the coarse levels, the pressure hierarchies) are bound by
// latency, not by the bytes the padding adds.
constexpr double kSellJagPadding = 1.10;
constexpr double kSellJagMinBytes = 32.0 * (1 << 20);

// Convert a BSR matrix (sorted rows) into sliced ELL of value type T, padded
// or jagged by the rule above.
template <typename T, typename TI>
Sell<T> to_sell(const BsrView<TI> &A, cudaStream_t s);

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

// Jagged slices (layout above): one warp per slice, the loop over the slots
// uniform across the warp; a lane loads only while its row has entries.
template <int BR, int BC, typename TA, typename TX, typename Epi>
__global__ void __launch_bounds__(256) k_sell_spmv_jag(SellView<TA> A, const TX *__restrict__ x, Epi epi) {
  constexpr int BS = BR * BC;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t slice = t / kSellH;
  const int lane = (int)(t % kSellH);
  if (slice >= A.nslice) return;   // whole warps: blockDim is a multiple of kSellH
  const int m = __ldg(A.lm + t);
  const int len = m >> 5;
  const int w = __shfl_sync(0xffffffffu, len, 0);   // lane 0 holds the longest row
  int64_t off = A.sp[slice];
  TA acc[BR];
#pragma unroll
  for (int q = 0; q < BR; q++) acc[q] = TA(0);
#pragma unroll 4
  for (int k = 0; k < w; k++) {
    const int ak = __popc(__ballot_sync(0xffffffffu, k < len));
    if (k < len) {
      const int c = __ldg(A.ci + off + lane);
      const TA *__restrict__ v = A.val + off * BS + lane;
      TA a[BS];
#pragma unroll
      for (int q = 0; q < BS; q++) a[q] = __ldg(v + (int64_t)q * ak);
      TA xv[BC];
#pragma unroll
      for (int j = 0; j < BC; j++) xv[j] = (TA)__ldg(x + (int64_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; r++)
#pragma unroll
        for (int j = 0; j < BC; j++) acc[r] += a[r * BC + j] * xv[j];
    }
    off += ak;
  }
  const int64_t out = slice * kSellH + (m & 31);
  if (out < A.nbr) epi(out, acc);
}

// Jagged lane-group slices, of one matrix or of two with the same rows and
// column space read in one pass (the prolongator P and the product S P of a
// V-cycle level, both applied to the coarse correction).  G lanes work on a
// row (G = 1, 4, 8, 16 or 32; a slice of 32 lanes holds 32 / G rows in
// natural order): lane j of a row takes its entries j, j + G, j + 2G, ... (for
// two matrices, the row's entries of the first, then those of the second).
// At slot k the lanes that still have an entry store theirs contiguously in
// lane order, a column index each and then each block scalar as one run of
// the active count; a lane finds its place as the popcount of the active
// lanes below it.  Every load a warp issues is then one contiguous run with
// no padding in it, however uneven the rows, and a slice starts at the sum of
// the row pointers of its first row.  Sums over a row's lanes are taken with
// shuffles, and the row's first lane runs the epilogue.
template <typename T>
struct JagView {
  int nbr = 0, nbc = 0, br = 0, bc = 0, nslice = 0, g = 1;
  const int64_t *sp = nullptr;   // nslice + 1 entry offsets
  const int2 *len = nullptr;     // per row: (entries of the first matrix, entries of both)
  const int *ci = nullptr;
  const T *val = nullptr;
};

template <typename T>
struct Jag {
  int nbr = 0, nbc = 0, br = 0, bc = 0, nslice = 0, g = 1;
  int64_t nnzb = 0;
  DBuf<int64_t> sp;
  DBuf<int2> len;
  DBuf<int> ci;
  DBuf<T> val;
  JagView<T> view() const {
    JagView<T> v;
    v.nbr = nbr; v.nbc = nbc; v.br = br; v.bc = bc; v.nslice = nslice; v.g = g;
    v.sp = sp.p; v.len = len.p; v.ci = ci.p; v.val = val.p;
    return v;
  }
};

// Lanes per row for a jagged layout with `per` entries per row on average:
// the fewest that leave a row at most kJagMaxSlots slots, then more while
// the launch would hold fewer than kJagMinWarps warps (32 per SM).  Measured
// on the fused prolongation at 128^3: one lane per row on the finest level
// (22 entries per row) and 4 on the first coarse level (42 per row) gave the
// shortest cycle; one lane everywhere made the coarse part 29% slower, and
// every rule with more lanes on the finest level made its pass slower.
#ifndef FS_JAG_MAX_SLOTS
#define FS_JAG_MAX_SLOTS 24.0
#endif
#ifndef FS_JAG_MIN_WARPS
#define FS_JAG_MIN_WARPS (32 * 152)
#endif
constexpr double kJagMaxSlots = FS_JAG_MAX_SLOTS;
constexpr int64_t kJagMinWarps = FS_JAG_MIN_WARPS;
inline int jag_lanes(int64_t nnzb, int nbr) {
  const double per = nbr > 0 ? (double)nnzb / nbr : 0.0;
  const int opts[5] = {1, 4, 8, 16, 32};
  int i = 0;
  while (i < 4 && per / opts[i] > kJagMaxSlots) i++;
  while (i < 4 && (int64_t)nbr * opts[i] / 32 < kJagMinWarps) i++;
  return opts[i];
}

// [P | Q] (Q null: P alone) of BSR matrices with equal rows, block shape and
// columns (P in double, Q in double or float), values in T, g lanes per row.
template <typename T, typename TQ>
Jag<T> to_jag(const BsrView<double> &P, const BsrView<TQ> *Q, int g, cudaStream_t s);

// one matrix: epi(row, acc); two: epi(row, acc1, acc2)
template <int BR, int BC, int G, bool TWO, typename TA, typename TX, typename Epi>
__global__ void __launch_bounds__(256) k_jag_spmv(JagView<TA> A, const TX *__restrict__ x, Epi epi) {
  constexpr int BS = BR * BC;
  constexpr int RPS = kSellH / G;   // rows per slice
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t slice = t / kSellH;
  const int lane = (int)(t % kSellH);
  if (slice >= A.nslice) return;   // whole warps: blockDim is a multiple of kSellH
  const int j = lane % G;
  const int64_t row = slice * RPS + lane / G;
  const int2 ln = row < A.nbr ? A.len[row] : make_int2(0, 0);
  int w = (ln.y + G - 1) / G;
#pragma unroll
  for (int o = kSellH / 2; o; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
  const unsigned below = (1u << lane) - 1u;
  int64_t off = A.sp[slice];
  TA a1[BR], a2[BR];
#pragma unroll
  for (int q = 0; q < BR; q++) a1[q] = a2[q] = TA(0);
#pragma unroll 2
  for (int k = 0; k < w; k++) {
    const int e = j + G * k;
    const bool on = e < ln.y;
    const unsigned act = __ballot_sync(0xffffffffu, on);
    const int ak = __popc(act);
    if (on) {
      const int rk = __popc(act & below);
      const int c = __ldg(A.ci + off + rk);
      const TA *__restrict__ v = A.val + off * BS + rk;
      TA a[BS];
#pragma unroll
      for (int q = 0; q < BS; q++) a[q] = __ldg(v + (int64_t)q * ak);
      TA xv[BC];
#pragma unroll
      for (int jj = 0; jj < BC; jj++) xv[jj] = (TA)__ldg(x + (int64_t)c * BC + jj);
      const bool first = !TWO || e < ln.x;
#pragma unroll
      for (int r = 0; r < BR; r++) {
        TA u = first ? a1[r] : a2[r];
#pragma unroll
        for (int jj = 0; jj < BC; jj++) u += a[r * BC + jj] * xv[jj];
        if (first) a1[r] = u;
        else a2[r] = u;
      }
    }
    off += ak;
  }
#pragma unroll
  for (int q = 0; q < BR; q++) {
    a1[q] = group_sum<G>(a1[q]);
    if constexpr (TWO) a2[q] = group_sum<G>(a2[q]);
  }
  if (row < A.nbr && j == 0) {
    if constexpr (TWO) epi(row, a1, a2);
    else epi(row, a1);
  }
}

template <int BR, int BC, bool TWO, typename TA, typename TX, typename Epi>
inline void jag_launch(const JagView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  if (A.nbr <= 0) return;
  const int threads = 256;
  const int64_t blocks = ((int64_t)A.nslice * kSellH + threads - 1) / threads;
  switch (A.g) {
    case 1: k_jag_spmv<BR, BC, 1, TWO, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    case 4: k_jag_spmv<BR, BC, 4, TWO, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    case 8: k_jag_spmv<BR, BC, 8, TWO, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    case 16: k_jag_spmv<BR, BC, 16, TWO, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
    default: k_jag_spmv<BR, BC, 32, TWO, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi); break;
  }
  FS_LAUNCHED();
}
template <int BR, int BC, typename TA, typename TX, typename Epi>
inline void jag2_spmv(const JagView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  jag_launch<BR, BC, true>(A, x, epi, s);
}

template <int BR, int BC, typename TA, typename TX, typename Epi>
inline void sell_spmv(const SellView<TA> &A, const TX *x, const Epi &epi, cudaStream_t s) {
  if (A.nbr <= 0) return;
  const int threads = 256;
  const int64_t blocks = ((int64_t)A.nslice * kSellH + threads - 1) / threads;
  if (A.lm) k_sell_spmv_jag<BR, BC, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi);
  else k_sell_spmv<BR, BC, TA, TX, Epi><<<(unsigned)blocks, threads, 0, s>>>(A, x, epi);
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
