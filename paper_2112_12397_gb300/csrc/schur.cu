// Setup of the approximate Schur complements (double precision).
//
//   H~ = Bdiag(H, 3) and its inverse           Alg. 1, Alg. 3
//   S1 = A + C1 H~^-1 C2                       Eq. Schur1_2, Alg. 3
//   S~ = S1 - Q1 T~^-1 Q2, T~ = diag(T)        Eq. appSchur_1, Alg. 1
//   S~2 = T - S_K                              Eq. app_Schur2_2, Alg. 3
//   [S_K]_k = Q2^(k)T (S1^(k))^-1 Q1^(k)       Eq. FS_algebraic (Remark rem:FS)
// S_K: for every face k with a nonzero row of Q2, the scalar index set
// K = nz(Q1 column k) U nz(Q2 row k) (entries that are exactly zero do not
// count) selects the principal submatrix S1^(k); one block per face gathers
// it into shared memory and solves with partial pivoting.
#include "schur.cuh"
#include "sparse.cuh"

namespace fs {

namespace {

__global__ void k_htilde_inv(BsrView<double> H, double *Hinv, int *flag) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < H.nbr;
       f += (int64_t)gridDim.x * blockDim.x) {
    int s = H.rp[f], len = H.rp[f + 1] - s;
    int p = find_sorted(H.ci + s, len, (int)f);
    double a[9];
    for (int k = 0; k < 9; k++) a[k] = p >= 0 ? H.val[(int64_t)(s + p) * 9 + k] : 0.0;
    double c00 = a[4] * a[8] - a[5] * a[7];
    double c01 = a[5] * a[6] - a[3] * a[8];
    double c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    double sc = 0.0;
    for (int k = 0; k < 9; k++) sc = fmax(sc, fabs(a[k]));
    double *o = Hinv + f * 9;
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

// X(i, f) = C1(i, f) * Hinv_f   (right scaling of each 3x3 block)
__global__ void k_scale_cols_3x3(BsrView<double> C, const double *Hinv, double *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < C.nnzb;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double *c = C.val + e * 9;
    const double *h = Hinv + (int64_t)C.ci[e] * 9;
    double *o = out + e * 9;
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 3; q++) {
        double s = 0.0;
        for (int t = 0; t < 3; t++) s += c[r * 3 + t] * h[t * 3 + q];
        o[r * 3 + q] = s;
      }
  }
}

__global__ void k_diag_scalar(BsrView<double> T, double *d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int s = T.rp[i], len = T.rp[i + 1] - s;
    int p = find_sorted(T.ci + s, len, (int)i);
    d[i] = p >= 0 ? T.val[s + p] : 0.0;
  }
}

// Y(i, k) = Q1(i, k) / T_kk   (3x1 blocks)
__global__ void k_scale_q1(BsrView<double> Q1, const double *tdiag, double *out, int *flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Q1.nnzb;
       e += (int64_t)gridDim.x * blockDim.x) {
    double t = tdiag[Q1.ci[e]];
    if (!(t != 0.0)) atomicExch(flag, 1);
    for (int r = 0; r < 3; r++) out[e * 3 + r] = Q1.val[e * 3 + r] / t;
  }
}

constexpr int kFsMax = 64;      // largest index set K^(k)
constexpr int kFsThreads = 128;

// one block per face: [S_K]_k
__global__ void __launch_bounds__(kFsThreads)
    k_fixed_stress(BsrView<double> S1, BsrView<double> Q1T, BsrView<double> Q2, double *SK, int *flag) {
  __shared__ double M[kFsMax * kFsMax];
  __shared__ double q1[kFsMax], q2[kFsMax];
  __shared__ int K[kFsMax];
  __shared__ int m_sh;
  for (int k = blockIdx.x; k < Q2.nbr; k += gridDim.x) {
    if (threadIdx.x == 0) {
      // gather K2 (Q2 row k) and K1 (Q1 column k = Q1^T row k), scalar indices
      int m = 0;
      bool ok = true, any2 = false;
      for (int e = Q2.rp[k]; e < Q2.rp[k + 1]; e++)
        for (int c = 0; c < 3; c++)
          if (Q2.val[(int64_t)e * 3 + c] != 0.0) any2 = true;
      if (any2) {
        for (int pass = 0; pass < 2 && ok; pass++) {
          const BsrView<double> &Q = pass == 0 ? Q2 : Q1T;
          for (int e = Q.rp[k]; e < Q.rp[k + 1] && ok; e++)
            for (int c = 0; c < 3; c++) {
              if (Q.val[(int64_t)e * 3 + c] == 0.0) continue;
              int idx = 3 * Q.ci[e] + c;
              int pos = m;
              bool dup = false;
              for (int t = 0; t < m; t++) dup |= (K[t] == idx);
              if (dup) continue;
              if (m >= kFsMax) { ok = false; break; }
              while (pos > 0 && K[pos - 1] > idx) { K[pos] = K[pos - 1]; pos--; }
              K[pos] = idx;
              m++;
            }
        }
      }
      if (!ok) { atomicExch(flag, 2); m = 0; }
      m_sh = any2 ? m : 0;
    }
    __syncthreads();
    const int m = m_sh;
    if (m == 0) {
      if (threadIdx.x == 0) SK[k] = 0.0;
      __syncthreads();
      continue;
    }
    // dense S1^(k), q1 = Q1[K, k], q2 = Q2[k, K]
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      int a = t / m, b = t - a * m;
      int ra = K[a] / 3, ca = K[a] - 3 * ra, rb = K[b] / 3, cb = K[b] - 3 * rb;
      int s = S1.rp[ra], len = S1.rp[ra + 1] - s;
      int p = find_sorted(S1.ci + s, len, rb);
      M[a * kFsMax + b] = p >= 0 ? S1.val[(int64_t)(s + p) * 9 + ca * 3 + cb] : 0.0;
    }
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
      int node = K[a] / 3, c = K[a] - 3 * node;
      double v1 = 0.0, v2 = 0.0;
      int s = Q1T.rp[k], len = Q1T.rp[k + 1] - s;
      int p = find_sorted(Q1T.ci + s, len, node);
      if (p >= 0) v1 = Q1T.val[(int64_t)(s + p) * 3 + c];
      s = Q2.rp[k]; len = Q2.rp[k + 1] - s;
      p = find_sorted(Q2.ci + s, len, node);
      if (p >= 0) v2 = Q2.val[(int64_t)(s + p) * 3 + c];
      q1[a] = v1;
      q2[a] = v2;
    }
    __syncthreads();
    // LU with partial pivoting (lowest index on ties), forward elimination on q1
    for (int j = 0; j < m; j++) {
      if (threadIdx.x == 0) {
        int p = j;
        double best = fabs(M[j * kFsMax + j]);
        for (int i = j + 1; i < m; i++) {
          double v = fabs(M[i * kFsMax + j]);
          if (v > best) { best = v; p = i; }
        }
        if (!(best > 0.0)) atomicExch(flag, 1);
        if (p != j) {
          for (int c = 0; c < m; c++) {
            double t = M[j * kFsMax + c];
            M[j * kFsMax + c] = M[p * kFsMax + c];
            M[p * kFsMax + c] = t;
          }
          double t = q1[j]; q1[j] = q1[p]; q1[p] = t;
        }
      }
      __syncthreads();
      const double pv = M[j * kFsMax + j];
      const int rows = m - j - 1;
      for (int t = threadIdx.x; t < rows * (m - j); t += blockDim.x) {
        int i = j + 1 + t / (m - j), c = j + t % (m - j);
        double l = M[i * kFsMax + j] / pv;
        if (c > j) M[i * kFsMax + c] -= l * M[j * kFsMax + c];
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
        double l = M[i * kFsMax + j] / pv;
        q1[i] -= l * q1[j];
        M[i * kFsMax + j] = l;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // back substitution and the product with q2
      for (int i = m - 1; i >= 0; i--) {
        double s = q1[i];
        for (int c = i + 1; c < m; c++) s -= M[i * kFsMax + c] * q1[c];
        q1[i] = s / M[i * kFsMax + i];
      }
      double sk = 0.0;
      for (int i = 0; i < m; i++) sk += q2[i] * q1[i];
      SK[k] = sk;
    }
    __syncthreads();
  }
}

// S~2 = T - diag(SK) on the pattern of T
__global__ void k_sub_diag(BsrView<double> T, const double *SK, double *val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T.nbr;
       i += (int64_t)gridDim.x * blockDim.x) {
    int s = T.rp[i], len = T.rp[i + 1] - s;
    int p = find_sorted(T.ci + s, len, (int)i);
    if (p >= 0) val[s + p] -= SK[i];
  }
}

inline int g(int64_t n) { return blocks_for(n, 256, kSMs * 16); }

// geometric fixed stress (Eq. FS): [S_K]_k = -omega_k / (kbar_k dt) on faces
// whose row of Q2 holds a nonzero entry, 0 elsewhere (the sign and the 1/dt
// of Q2 = -Q1^T / dt on open faces)
__global__ void k_fixed_stress_geometric(BsrView<double> Q2, const double *omega, const double *kbar,
                                         double dt, double *SK) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Q2.nbr;
       k += (int64_t)gridDim.x * blockDim.x) {
    bool nz = false;
    for (int e = Q2.rp[k]; e < Q2.rp[k + 1] && !nz; e++)
      for (int q = 0; q < 3; q++) nz |= Q2.val[(int64_t)e * 3 + q] != 0.0;
    SK[k] = nz ? -omega[k] / (kbar[k] * dt) : 0.0;
  }
}

}  // namespace

void build_hinv(const BsrView<double> &H, DBuf<double> &Hinv, cudaStream_t s) {
  Hinv.alloc((size_t)H.nbr * 9 > 0 ? (size_t)H.nbr * 9 : 1);
  if (H.nbr == 0) return;
  DBuf<int> flag(1);
  FS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  k_htilde_inv<<<g(H.nbr), 256, 0, s>>>(H, Hinv.p, flag.p);
  FS_LAUNCHED();
  int h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!h, FC_SINGULAR_BLOCK, "singular 3x3 diagonal block of H (H~ = Bdiag(H,3))");
}

Bsr<double> build_s1(const BsrView<double> &A, const BsrView<double> &C1, const BsrView<double> &C2,
                     const double *Hinv, cudaStream_t s) {
  Bsr<double> X;
  X.shape(C1.nbr, C1.nbc, 3, 3);
  X.nnzb = C1.nnzb;
  X.rp.alloc(C1.nbr + 1);
  X.ci.alloc(C1.nnzb);
  X.val.alloc(C1.nnzb * 9);
  FS_CUDA(cudaMemcpyAsync(X.rp.p, C1.rp, sizeof(int) * (C1.nbr + 1), cudaMemcpyDeviceToDevice, s));
  if (C1.nnzb) {
    FS_CUDA(cudaMemcpyAsync(X.ci.p, C1.ci, sizeof(int) * C1.nnzb, cudaMemcpyDeviceToDevice, s));
    k_scale_cols_3x3<<<g(C1.nnzb), 256, 0, s>>>(C1, Hinv, X.val.p);
    FS_LAUNCHED();
  }
  Bsr<double> Y = spgemm(X.view(), C2, s);
  return spadd(A, Y.view(), 1.0, 1.0, s);
}

Bsr<double> build_stilde(const BsrView<double> &S1, const BsrView<double> &Q1, const BsrView<double> &Q2,
                         const BsrView<double> &T, cudaStream_t s) {
  DBuf<double> td(T.nbr > 0 ? T.nbr : 1);
  if (T.nbr) {
    k_diag_scalar<<<g(T.nbr), 256, 0, s>>>(T, td.p);
    FS_LAUNCHED();
  }
  Bsr<double> Y;
  Y.shape(Q1.nbr, Q1.nbc, 3, 1);
  Y.nnzb = Q1.nnzb;
  Y.rp.alloc(Q1.nbr + 1);
  Y.ci.alloc(Q1.nnzb);
  Y.val.alloc(Q1.nnzb * 3);
  FS_CUDA(cudaMemcpyAsync(Y.rp.p, Q1.rp, sizeof(int) * (Q1.nbr + 1), cudaMemcpyDeviceToDevice, s));
  DBuf<int> flag(1);
  FS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  if (Q1.nnzb) {
    FS_CUDA(cudaMemcpyAsync(Y.ci.p, Q1.ci, sizeof(int) * Q1.nnzb, cudaMemcpyDeviceToDevice, s));
    k_scale_q1<<<g(Q1.nnzb), 256, 0, s>>>(Q1, td.p, Y.val.p, flag.p);
    FS_LAUNCHED();
  }
  int h = 0;
  FS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  FS_CUDA(cudaStreamSynchronize(s));
  FS_REQUIRE(!h, FC_SINGULAR_BLOCK, "zero diagonal entry of T");
  Bsr<double> Z = spgemm(Y.view(), Q2, s);
  return spadd(S1, Z.view(), 1.0, -1.0, s);
}

Bsr<double> build_s2tilde(const BsrView<double> &S1, const BsrView<double> &Q1, const BsrView<double> &Q2,
                          const BsrView<double> &T, DBuf<double> &SK, cudaStream_t s, const GeoFs *geo) {
  const int nf = Q2.nbr;
  SK.alloc(nf > 0 ? nf : 1);
  if (geo && geo->omega) {
    if (nf) {
      k_fixed_stress_geometric<<<g(nf), 256, 0, s>>>(Q2, geo->omega, geo->kbar, geo->dt, SK.p);
      FS_LAUNCHED();
    }
  } else {
    Bsr<double> Q1T = transpose(Q1, s);
    DBuf<int> flag(1);
    FS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
    if (nf) {
      k_fixed_stress<<<kSMs * 16, kFsThreads, 0, s>>>(S1, Q1T.view(), Q2, SK.p, flag.p);
      FS_LAUNCHED();
    }
    int h = 0;
    FS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    FS_REQUIRE(h != 2, FC_INTERNAL, "fixed-stress index set larger than 64");
    FS_REQUIRE(h != 1, FC_SINGULAR_BLOCK, "singular local block S1^(k) in the fixed-stress diagonal");
  }
  Bsr<double> S2 = copy_cast<double, double>(T, s);
  if (nf) {
    k_sub_diag<<<g(nf), 256, 0, s>>>(T, SK.p, S2.val.p);
    FS_LAUNCHED();
  }
  FS_CUDA(cudaStreamSynchronize(s));
  return S2;
}

}  // namespace fs
