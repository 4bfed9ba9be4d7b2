// Approximate Schur complements of Alg. 1 and Alg. 3 (setup, double).
#pragma once

#include "common.cuh"

namespace fs {

// H~^-1: inverse of the 3x3 diagonal block of every face row of H.
void build_hinv(const BsrView<double> &H, DBuf<double> &Hinv, cudaStream_t s);

// S1 = A + C1 H~^-1 C2.
Bsr<double> build_s1(const BsrView<double> &A, const BsrView<double> &C1, const BsrView<double> &C2,
                     const double *Hinv, cudaStream_t s);

// S~ = S1 - Q1 diag(T)^-1 Q2.
Bsr<double> build_stilde(const BsrView<double> &S1, const BsrView<double> &Q1, const BsrView<double> &Q2,
                         const BsrView<double> &T, cudaStream_t s);

// Data of the geometric fixed stress (Eq. FS): per face the volume of the
// cells around it and their bulk modulus (device arrays), and the time step.
struct GeoFs {
  const double *omega = nullptr;
  const double *kbar = nullptr;
  double dt = 0.0;
};

// S~2 = T - S_K (written to SK) with the algebraic fixed-stress diagonal
// (Eq. FS_algebraic), or the geometric one when geo carries data.
Bsr<double> build_s2tilde(const BsrView<double> &S1, const BsrView<double> &Q1, const BsrView<double> &Q2,
                          const BsrView<double> &T, DBuf<double> &SK, cudaStream_t s,
                          const GeoFs *geo = nullptr);

}  // namespace fs
