// Sparse matrix construction on the device (setup phase, double precision):
// transpose, block SpGEMM (hash symbolic + Gustavson numeric), sparse add.
#pragma once

#include "common.cuh"
#include "spmv.cuh"

namespace fs {

// Position of `col` in the sorted column list ci[0..n), or -1.
__device__ inline int find_sorted(const int *ci, int n, int col) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int c = ci[mid];
    if (c == col) return mid;
    if (c < col) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// A^T with transposed blocks; rows of the result sorted by column.
Bsr<double> transpose(const BsrView<double> &A, cudaStream_t s);

// C = A B for block shapes (A.br x A.bc) (B.br x B.bc), A.bc == B.br.
// Supported shapes: 3x3*3x3, 3x1*1x3, 1x1*1x1, 3x3*3x1, 1x3*3x3.
// Rows of C sorted; entries that cancel to zero are kept.  T = double or
// float (the products and sums in T; the same pattern and summation order).
template <typename T>
Bsr<T> spgemm(const BsrView<T> &A, const BsrView<T> &B, cudaStream_t s);

// Numeric pass only: C (whose pattern is that of A B, e.g. from an earlier
// spgemm of the same patterns) receives the values of A B.
template <typename T>
void spgemm_numeric(const BsrView<T> &A, const BsrView<T> &B, Bsr<T> &C, cudaStream_t s);

// True when the n doubles at a and b are bitwise identical (device arrays).
bool same_values(const double *a, const double *b, int64_t n, cudaStream_t s);

// Validates a caller's block structure on the device before any kernel
// indexes through it: 0 = valid; bit 1 = row pointers not 0 .. nnzb
// non-decreasing; bit 2 = a column outside [0, nbc) or not strictly
// increasing within its row (checked only when the row pointers are valid).
int check_structure(const BsrView<double> &A, cudaStream_t s);

// True when A and B have identical row pointers and column indices.
bool same_pattern(const BsrView<double> &A, const BsrView<double> &B, cudaStream_t s);

// C = alpha A + beta B (same shape and block size), rows sorted.
Bsr<double> spadd(const BsrView<double> &A, const BsrView<double> &B, double alpha, double beta,
                  cudaStream_t s);

// Deep copy of a BSR view into an owned matrix (same value type).
template <typename TO, typename TI>
Bsr<TO> copy_cast(const BsrView<TI> &A, cudaStream_t s);

// Chunked copy (values cast to T) of a BSR matrix with g lanes per row.
template <typename T>
Chunked<T> to_chunked(const BsrView<double> &A, int g, cudaStream_t s);

// Upload a host BSR (double) into an owned device matrix.
Bsr<double> upload_bsr(int nbr, int nbc, int br, int bc, int64_t nnzb, const int *rp_dev,
                       const int *ci_dev, const double *val_dev, cudaStream_t s);

// Download to host vectors.
void download_bsr(const BsrView<double> &A, std::vector<int> &rp, std::vector<int> &ci,
                  std::vector<double> &val, cudaStream_t s);

}  // namespace fs
