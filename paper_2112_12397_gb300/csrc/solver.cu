// The C-ABI of libfracsolve: setup of the block preconditioners (Alg. 1, 3),
// their application (Alg. 2, 4), the Jacobian product (Eq. JacSys) and the
// right-preconditioned flexible GMRES with CGS2 of Sec. 4.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <type_traits>

#include "amg.cuh"
#include "schur.cuh"
#include "sell.cuh"
#include "sparse.cuh"
#include "spmv.cuh"

using namespace fs;

namespace {

template <typename TP>
struct PrecData {
  BsrView<TP> C1, Q1, C2, Q2;
  const TP *Hinv = nullptr;
  Bsr<TP> C1o, Q1o, C2o, Q2o;
  DBuf<TP> Hinvo;
  Sell<TP> sC1, sQ1, sC2, sQ2;   // sliced-ELL copies used by the products
  Sell<TP> tC1, tQ1, tC2, tQ2;   // transposes, for the adjoint preconditioner
  DBuf<TP> HinvT;                // transposed H~^-1 blocks
  bool ready_t = false;
  DBuf<TP> w, out, tt, tu, su, tp, sp, vp;
  bool ready = false;
};

// ------------------------------------------------------------ small kernels
template <typename TP>
__global__ void k_face_hinv(int64_t nf, const TP *Hinv, const TP *in, TP *out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    const TP *h = Hinv + f * 9;
    TP a = in[3 * f], b = in[3 * f + 1], c = in[3 * f + 2];
    out[3 * f] = h[0] * a + h[1] * b + h[2] * c;
    out[3 * f + 1] = h[3] * a + h[4] * b + h[5] * c;
    out[3 * f + 2] = h[6] * a + h[7] * b + h[8] * c;
  }
}

// out = Hinv in per face, and neg = -out (the t block of D2^-1 L2^-1)
template <typename TP>
__global__ void k_face_hinv_neg(int64_t nf, const TP *Hinv, const TP *in, TP *out, TP *neg) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    const TP *h = Hinv + f * 9;
    TP a = in[3 * f], b = in[3 * f + 1], c = in[3 * f + 2];
    const TP o0 = h[0] * a + h[1] * b + h[2] * c;
    const TP o1 = h[3] * a + h[4] * b + h[5] * c;
    const TP o2 = h[6] * a + h[7] * b + h[8] * c;
    out[3 * f] = o0; out[3 * f + 1] = o1; out[3 * f + 2] = o2;
    neg[3 * f] = -o0; neg[3 * f + 1] = -o1; neg[3 * f + 2] = -o2;
  }
}

// x = sum_j Z_j y_j
template <typename TP>
__global__ void k_mcomb(const TP *__restrict__ Z, int k, int64_t n, const double *__restrict__ y, double *x) {
  extern __shared__ double ys[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; j++) s += (double)Z[(int64_t)j * n + e] * ys[j];
    x[e] = s;
  }
}

// Classical Gram-Schmidt passes over the basis V (m vectors of length n,
// row-major).  Both kernels are bound by the FP64 FMA rate rather than by
// HBM on this part, so they are laid out for arithmetic throughput: the dot
// kernel sweeps the vector with a grid of 8 blocks per SM, kCgsQ basis
// vectors per sweep (w is re-read per sweep from L2), and reduces per block
// into partial sums that a second kernel adds in a fixed order; the update
// kernel gives each thread one entry of w and all m basis vectors.
constexpr int kCgsT = 256, kCgsQ = 4;
constexpr int kCgsDotGrid = kSMs * 8, kCgsSubGrid = kSMs * 16;

// partial[i * gridDim.x + block] = V_i . w over the block's entries (i < m);
// with_norm adds row m = w . w
__global__ void __launch_bounds__(kCgsT)
    k_cgs_dot(const double *__restrict__ V, int m, int64_t n, const double *__restrict__ w, double *partial,
              int with_norm) {
  __shared__ double red[kCgsT / 32][kCgsQ];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int mm = m + (with_norm ? 1 : 0);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int i0 = 0; i0 < mm; i0 += kCgsQ) {
    const int nq = min(kCgsQ, mm - i0);
    double acc[kCgsQ];
#pragma unroll
    for (int q = 0; q < kCgsQ; q++) acc[q] = 0.0;
#pragma unroll 2
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + tid; e < n; e += stride) {
      const double we = __ldg(w + e);
#pragma unroll
      for (int q = 0; q < kCgsQ; q++)
        if (q < nq) {
          const int i = i0 + q;
          const double v = i < m ? __ldg(V + (int64_t)i * n + e) : we;
          acc[q] += v * we;
        }
    }
#pragma unroll
    for (int q = 0; q < kCgsQ; q++) {
      const double r = warp_sum(acc[q]);
      if (lane == 0) red[wid][q] = r;
    }
    __syncthreads();
    if (tid < nq) {
      double sum = 0.0;
#pragma unroll
      for (int k = 0; k < kCgsT / 32; k++) sum += red[k][tid];
      partial[(int64_t)(i0 + tid) * gridDim.x + blockIdx.x] = sum;
    }
    __syncthreads();
  }
}

// h[i] = sum_b partial[i][b] (fixed order); hacc[i] (+)= h[i] for i < m;
// row m (if present) goes to *extra
__global__ void k_cgs_final(const double *partial, int m, int rows, int nb, double *h, double *hacc,
                            int accumulate, double *extra) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += (gridDim.x * blockDim.x) >> 5) {
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += partial[(int64_t)i * nb + b];
    v = warp_sum(v);
    if (lane == 0) {
      if (i < m) {
        h[i] = v;
        hacc[i] = accumulate ? hacc[i] + v : v;
      } else {
        *extra = v;
      }
    }
  }
}

// w -= V h, one thread per entry; partial_norm (if given): partial[block] =
// the block's share of ||w||^2 after the update
__global__ void __launch_bounds__(kCgsT)
    k_cgs_sub(const double *__restrict__ V, int m, int64_t n, const double *__restrict__ h, double *w,
              double *partial_norm) {
  extern __shared__ double hs[];
  __shared__ double red[kCgsT / 32];
  for (int i = threadIdx.x; i < m; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double nn = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + tid; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
#pragma unroll 8
    for (int i = 0; i < m; i++) sum += __ldg(V + (int64_t)i * n + e) * hs[i];
    const double we = w[e] - sum;
    w[e] = we;
    nn += we * we;
  }
  if (partial_norm) {
    nn = warp_sum(nn);
    if (lane == 0) red[wid] = nn;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int k = 0; k < kCgsT / 32; k++) sum += red[k];
      partial_norm[blockIdx.x] = sum;
    }
  }
}

// Arnoldi column j: Hessenberg entries from hacc and ||w||^2, previous Givens
// rotations, a new rotation, the residual recurrence.  stat[0] = |g_{j+1}|/beta,
// stat[1] = h_{j+1,j}, stat[2] = w0 (norm before orthogonalisation),
// stat[3] = 1 / h_{j+1,j} (0 on breakdown).
__global__ void k_givens(int j, int ld, const double *hacc, const double *w2, const double *w02, double beta,
                         double *Hm, double *cs, double *sn, double *g, double *stat) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double *col = Hm + (int64_t)j * ld;
  for (int i = 0; i <= j; i++) col[i] = hacc[i];
  const double hn = sqrt(*w2);
  const double w0 = sqrt(*w02);
  col[j + 1] = hn;
  for (int i = 0; i < j; i++) {
    double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  double r = hypot(col[j], col[j + 1]);
  cs[j] = col[j] / r;
  sn[j] = col[j + 1] / r;
  col[j] = r;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  stat[0] = fabs(g[j + 1]) / beta;
  stat[1] = hn;
  stat[2] = w0;
  stat[3] = (hn > 1e-14 * w0 && hn > 0.0) ? 1.0 / hn : 0.0;
}

__global__ void k_scale_by(double *v, int64_t n, const double *sc) {
  const double a = *sc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    v[e] *= a;
}

__global__ void k_trisolve(int k, int ld, const double *Hm, const double *g, double *y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; i--) {
    double s = g[i];
    for (int c = i + 1; c < k; c++) s -= Hm[(int64_t)c * ld + i] * y[c];
    y[i] = s / Hm[(int64_t)i * ld + i];
  }
}

__global__ void k_set_scalar(double *p, double v) { *p = v; }

inline int vgrid(int64_t n) { return blocks_for(n, 256, kSMs * 16); }

}  // namespace

// ============================================================ context
struct fc_ctx {
  BlockCache cache;   // first member: destroyed after every buffer that returns to it
  fc_options opt;
  cudaStream_t s = nullptr;
  int device = 0;
  std::string err;
  bool ready = false;
  int nn = 0, nf = 0;
  int64_t n = 0, nu = 0, nt = 0;
  Bsr<double> A, C1, Q1, C2, H, Q2, T;
  Sell<double> sA, sC1, sQ1, sC2, sH, sQ2, sT;   // sliced-ELL copies for J z
  Sell<double> tA, tC1, tQ1, tC2, tH, tQ2, tT;   // transposed blocks for J^T z
  bool have_adj = false;
  DBuf<double> Hinv64, SK;
  Bsr<double> S1, St, S2t;
  bool have[2] = {false, false};
  Hierarchy hier[4];
  PrecData<float> pf;
  PrecData<double> pd;
  // Krylov workspace
  int kcap = 0;          // iterations the Krylov workspace holds ...
  int64_t kn = 0;        // ... for vectors of this length
  int kprec = -1;        // ... in this precision mode
  int kbasis = 0;        // orthonormal vectors of V left by the last FGMRES cycle
  DBuf<double> V, Hm, cs, sn, g, y, hacc, htmp, partial, stat, w2, w02, red;
  DBuf<float> Zf;
  DBuf<double> Zd;
  DBuf<double> xk, rk, bk, hb, hx;
  DBuf<double> zd;   // a float direction widened to double for J z / J^T z
  DBuf<double> geo_omega, geo_kbar;   // geometric fixed stress data (empty: algebraic)
  GeoFs geo;
  int64_t geo_n = 0;
  double *stat_host = nullptr;   // pinned
  Profiler prof;
  ~fc_ctx() {
    if (stat_host) cudaFreeHost(stat_host);
  }
};

namespace {

bool valid_variant(int v) { return v == FC_TPU || v == FC_TUP || v == FC_TUP_STAR; }

// the incomplete t-u-p form uses the t-u-p setup (S1, S~2 and their AMG)
bool built(const fc_ctx &c, int v) { return c.have[v == FC_TUP_STAR ? FC_TUP : v]; }

AmgParams amg_params(const fc_options &o, bool pressure) {
  AmgParams p;
  p.theta0 = o.theta0;
  p.theta_decay = o.theta_decay;
  p.coarse_max = pressure ? o.coarse_max_p : o.coarse_max;
  p.max_levels = o.max_levels;
  p.max_ratio = o.max_ratio;
  p.power_steps = o.power_steps;
  p.omega_num = o.omega_num;
  p.cheb_degree = o.cheb_degree;
  p.cheb_hi = o.cheb_hi;
  p.cheb_lo = o.cheb_lo;
  p.seed = o.amg_seed;
  p.verbose = o.verbose;
  p.graphs = o.coarse_graphs != 0;
  return p;
}

void check_bsr(const fc_bsr &m, int nbr, int nbc, int br, int bc, const char *name, cudaStream_t s) {
  bool ok = m.n_brows == nbr && m.n_bcols == nbc && m.br == br && m.bc == bc && m.nnzb >= 0 &&
            (m.nnzb == 0 || (m.d_col_idx && m.d_val)) && m.d_row_ptr;
  FS_REQUIRE(ok, FC_BAD_ARG, std::string("block ") + name + " has inconsistent sizes or null pointers");
  BsrView<double> v;
  v.nbr = m.n_brows; v.nbc = m.n_bcols; v.br = m.br; v.bc = m.bc; v.nnzb = m.nnzb;
  v.rp = m.d_row_ptr; v.ci = m.d_col_idx; v.val = m.d_val;
  const int bad = check_structure(v, s);
  FS_REQUIRE(!(bad & 1), FC_BAD_ARG,
             std::string("block ") + name + ": row pointers must run from 0 to nnzb without decreasing");
  FS_REQUIRE(!(bad & 2), FC_BAD_ARG,
             std::string("block ") + name + ": columns must lie in [0, n_bcols) and increase within each row");
}

template <typename TP>
void prepare_prec(fc_ctx &c, PrecData<TP> &P) {
  cudaStream_t s = c.s;
  if constexpr (std::is_same<TP, double>::value) {
    P.C1 = c.C1.view(); P.Q1 = c.Q1.view(); P.C2 = c.C2.view(); P.Q2 = c.Q2.view();
    P.Hinv = c.Hinv64.p;
  } else {
    P.C1o = copy_cast<TP, double>(c.C1.view(), s);
    P.Q1o = copy_cast<TP, double>(c.Q1.view(), s);
    P.C2o = copy_cast<TP, double>(c.C2.view(), s);
    P.Q2o = copy_cast<TP, double>(c.Q2.view(), s);
    P.C1 = P.C1o.view(); P.Q1 = P.Q1o.view(); P.C2 = P.C2o.view(); P.Q2 = P.Q2o.view();
    P.Hinvo.alloc((size_t)c.nf * 9 > 0 ? (size_t)c.nf * 9 : 1);
    cast(P.Hinvo.p, c.Hinv64.p, (int64_t)c.nf * 9, s);
    P.Hinv = P.Hinvo.p;
  }
  P.sC1 = to_sell<TP>(c.C1.view(), s);
  P.sQ1 = to_sell<TP>(c.Q1.view(), s);
  P.sC2 = to_sell<TP>(c.C2.view(), s);
  P.sQ2 = to_sell<TP>(c.Q2.view(), s);
  const int64_t n = c.n;
  P.w.alloc(n); P.out.alloc(n);
  P.tt.alloc(c.nt > 0 ? c.nt : 1);
  P.tu.alloc(c.nu); P.su.alloc(c.nu);
  P.tp.alloc(c.nf > 0 ? c.nf : 1); P.sp.alloc(c.nf > 0 ? c.nf : 1); P.vp.alloc(c.nf > 0 ? c.nf : 1);
  P.ready = true;
}

// z = M^-1 w, both in precision TP (Alg. 2, Alg. 4, or the incomplete
// t-u-p form D2^-1 L2^-1 of Eq. P2)
template <typename TP>
void apply_prec(fc_ctx &c, PrecData<TP> &P, int variant, const TP *w, TP *z) {
  NvtxRange nvtx("apply_prec");
  cudaStream_t s = c.s;
  const int64_t nu = c.nu, nt = c.nt;
  const int64_t nf = c.nf;
  const TP *w_u = w, *w_t = w + nu, *w_p = w + nu + nt;
  TP *z_u = z, *z_t = z + nu, *z_p = z + nu + nt;
  if (variant == FC_TUP_STAR) {
    Hierarchy &Hu = c.hier[FC_H_TUP_U], &Hp = c.hier[FC_H_TUP_P];
    if (nf) {   // t_t = H~^-1 w_t; v_t = -t_t
      k_face_hinv_neg<TP><<<vgrid(nf), 256, 0, s>>>(nf, P.Hinv, w_t, P.tt.p, z_t);
      FS_LAUNCHED();
    }
    sell_axpby<3, 3>(P.sC1.view(), P.tt.p, P.tu.p, 1.0, 1.0, w_u, s);   // y_u = w_u + C1 t_t
    c.prof.start(PK_VCYCLE, s);
    amg_vcycle<TP>(Hu, P.tu.p, z_u, s);                                  // v_u = S~1^-1 y_u
    c.prof.stop(PK_VCYCLE, s, 0.0);
    if (nf) {
      sell_axpby<1, 3>(P.sQ2.view(), z_u, P.tp.p, -1.0, 1.0, w_p, s);   // y_p = w_p - Q2 v_u
      c.prof.start(PK_VCYCLE_P, s);
      amg_vcycle<TP>(Hp, P.tp.p, z_p, s);                                // v_p = S~2^-1 y_p
      c.prof.stop(PK_VCYCLE_P, s, 0.0);
    }
  } else if (variant == FC_TUP) {
    Hierarchy &Hu = c.hier[FC_H_TUP_U], &Hp = c.hier[FC_H_TUP_P];
    if (nf) { k_face_hinv<TP><<<vgrid(nf), 256, 0, s>>>(nf, P.Hinv, w_t, P.tt.p); FS_LAUNCHED(); }   // t_t = H~^-1 w_t
    sell_axpby<3, 3>(P.sC1.view(), P.tt.p, P.tu.p, 1.0, 1.0, w_u, s);                                // t_u = w_u + C1 t_t
    c.prof.start(PK_VCYCLE, s);
    amg_vcycle<TP>(Hu, P.tu.p, P.su.p, s);                                                            // s_u = AMG(S1, t_u)
    c.prof.stop(PK_VCYCLE, s, 0.0);
    sell_axpby<1, 3>(P.sQ2.view(), P.su.p, P.tp.p, -1.0, 1.0, w_p, s);                              // t_p = w_p - Q2 s_u
    c.prof.start(PK_VCYCLE_P, s);
    if (nf) amg_vcycle<TP>(Hp, P.tp.p, z_p, s);                                                        // v_p = S~2^-1 t_p
    c.prof.stop(PK_VCYCLE_P, s, 0.0);
    sell_axpby<3, 1>(P.sQ1.view(), z_p, P.tu.p, 1.0, 0.0, (const TP *)nullptr, s);                 // t_u = Q1 v_p
    amg_vcycle<TP>(Hu, P.tu.p, z_u, s);                                                               // v_u = AMG(S1, t_u)
    axpbyz(z_u, P.su.p, z_u, 1.0, -1.0, nu, s);                                                       // v_u = s_u - v_u
    if (nf) {                                                                                         // v_t = -t_t + H~^-1 C2 v_u
      EpiHinvUpdate<TP> e{z_t, P.tt.p, P.Hinv};
      sell_spmv<3, 3>(P.sC2.view(), z_u, e, s);
    }
  } else {
    Hierarchy &Hu = c.hier[FC_H_TPU_U], &Hp = c.hier[FC_H_TPU_P];
    if (nf) amg_vcycle<TP>(Hp, w_p, P.tp.p, s);                                                        // t_p = T^-1 w_p
    if (nf) { k_face_hinv<TP><<<vgrid(nf), 256, 0, s>>>(nf, P.Hinv, w_t, P.tt.p); FS_LAUNCHED(); }    // t_t = H~^-1 w_t
    sell_axpby<3, 3>(P.sC1.view(), P.tt.p, P.tu.p, 1.0, 1.0, w_u, s);                                // t_u = w_u + C1 t_t - Q1 t_p
    sell_axpby<3, 1>(P.sQ1.view(), P.tp.p, P.tu.p, -1.0, 1.0, P.tu.p, s);
    amg_vcycle<TP>(Hu, P.tu.p, z_u, s);                                                               // v_u = AMG(S~, t_u)
    if (nf) {
      sell_axpby<1, 3>(P.sQ2.view(), z_u, P.sp.p, 1.0, 0.0, (const TP *)nullptr, s);                // s_p = Q2 v_u
      amg_vcycle<TP>(Hp, P.sp.p, P.vp.p, s);                                                          // v_p = t_p - T^-1 s_p
      axpbyz(z_p, P.tp.p, P.vp.p, 1.0, -1.0, nf, s);
      EpiHinvUpdate<TP> e{z_t, P.tt.p, P.Hinv};                                                      // v_t = -t_t + H~^-1 C2 v_u
      sell_spmv<3, 3>(P.sC2.view(), z_u, e, s);
    }
  }
}

// y = J z (double out)
template <typename T>
double bsr_bytes(const Bsr<double> &m) {
  return (double)m.nnzb * (m.br * m.bc * sizeof(T) + 4) + (double)(m.nbr + 1) * 4;
}

template <typename TX>
void jac_spmv(fc_ctx &c, const TX *z, double *y) {
  NvtxRange nvtx("J z");
  cudaStream_t s = c.s;
  const double bytes = bsr_bytes<double>(c.A) + bsr_bytes<double>(c.C1) + bsr_bytes<double>(c.Q1) +
                       bsr_bytes<double>(c.C2) + bsr_bytes<double>(c.H) + bsr_bytes<double>(c.Q2) +
                       bsr_bytes<double>(c.T) + (double)c.n * (sizeof(TX) + sizeof(double));
  c.prof.start(PK_JAC, s);
  // a float direction (mixed mode) is widened once: the products then run
  // entirely in FP64 FMAs, without a float-to-double conversion per block
  // (those occupy the same FP64 pipe as the FMAs)
  const double *zz;
  if constexpr (std::is_same<TX, float>::value) {
    c.zd.ensure(c.n);
    cast(c.zd.p, z, c.n, s);
    zz = c.zd.p;
  } else {
    zz = z;
  }
  const double *z_u = zz, *z_t = zz + c.nu, *z_p = zz + c.nu + c.nt;
  double *y_u = y, *y_t = y + c.nu, *y_p = y + c.nu + c.nt;
  sell_axpby<3, 3>(c.sA.view(), z_u, y_u, 1.0, 0.0, (const double *)nullptr, s);
  if (c.nf) {
    sell_axpby<3, 3>(c.sC1.view(), z_t, y_u, 1.0, 1.0, y_u, s);
    sell_axpby<3, 1>(c.sQ1.view(), z_p, y_u, 1.0, 1.0, y_u, s);
    sell_axpby<3, 3>(c.sC2.view(), z_u, y_t, 1.0, 0.0, (const double *)nullptr, s);
    sell_axpby<3, 3>(c.sH.view(), z_t, y_t, -1.0, 1.0, y_t, s);
    sell_axpby<1, 3>(c.sQ2.view(), z_u, y_p, 1.0, 0.0, (const double *)nullptr, s);
    sell_axpby<1, 1>(c.sT.view(), z_p, y_p, 1.0, 1.0, y_p, s);
  }
  c.prof.stop(PK_JAC, s, bytes);
}

// y = J^T z (double out): rows u [A^T C2^T Q2^T], rows t [C1^T -H^T 0],
// rows p [Q1^T 0 T^T]
template <typename TX>
void jac_spmv_t(fc_ctx &c, const TX *z, double *y) {
  cudaStream_t s = c.s;
  const double *zz;
  if constexpr (std::is_same<TX, float>::value) {
    c.zd.ensure(c.n);
    cast(c.zd.p, z, c.n, s);
    zz = c.zd.p;
  } else {
    zz = z;
  }
  const double *z_u = zz, *z_t = zz + c.nu, *z_p = zz + c.nu + c.nt;
  double *y_u = y, *y_t = y + c.nu, *y_p = y + c.nu + c.nt;
  sell_axpby<3, 3>(c.tA.view(), z_u, y_u, 1.0, 0.0, (const double *)nullptr, s);
  if (c.nf) {
    sell_axpby<3, 3>(c.tC2.view(), z_t, y_u, 1.0, 1.0, y_u, s);
    sell_axpby<3, 1>(c.tQ2.view(), z_p, y_u, 1.0, 1.0, y_u, s);
    sell_axpby<3, 3>(c.tC1.view(), z_u, y_t, 1.0, 0.0, (const double *)nullptr, s);
    sell_axpby<3, 3>(c.tH.view(), z_t, y_t, -1.0, 1.0, y_t, s);
    sell_axpby<1, 3>(c.tQ1.view(), z_u, y_p, 1.0, 0.0, (const double *)nullptr, s);
    sell_axpby<1, 1>(c.tT.view(), z_p, y_p, 1.0, 1.0, y_p, s);
  }
}

// z = M^-T w in precision TP: the transposed block factorisations of Eq. P1 /
// Eq. P2 applied in reverse order (transposed V-cycles for S~ / S1; T and
// S~2 are symmetric and so are their scalar V-cycles)
template <typename TP>
void apply_prec_t(fc_ctx &c, PrecData<TP> &P, int variant, const TP *w, TP *z) {
  NvtxRange nvtx("apply_prec_t");
  cudaStream_t s = c.s;
  const int64_t nu = c.nu, nt = c.nt, nf = c.nf;
  const TP *w_u = w, *w_t = w + nu, *w_p = w + nu + nt;
  TP *z_u = z, *z_t = z + nu, *z_p = z + nu + nt;
  if (variant == FC_TUP_STAR) {
    // (D2^-1 L2^-1)^T = L2^-T D2^-T: z_p = S~2^-T w_p; v_u = S~1^-T w_u -
    // S~1^-T Q2^T z_p, formed as one transposed V-cycle on w_u - Q2^T z_p
    // (the V-cycle is a fixed linear operator); v_t = H~^-T (C1^T v_u - w_t)
    Hierarchy &Hu = c.hier[FC_H_TUP_U], &Hp = c.hier[FC_H_TUP_P];
    if (nf) {
      amg_vcycle<TP>(Hp, w_p, z_p, s);
      sell_axpby<3, 1>(P.tQ2.view(), z_p, P.tu.p, -1.0, 1.0, w_u, s);
    }
    amg_vcycle_t<TP>(Hu, nf ? P.tu.p : w_u, z_u, s);
    if (nf) {
      k_face_hinv<TP><<<vgrid(nf), 256, 0, s>>>(nf, P.HinvT.p, w_t, P.tt.p);
      FS_LAUNCHED();
      EpiHinvUpdate<TP> e{z_t, P.tt.p, P.HinvT.p};
      sell_spmv<3, 3>(P.tC1.view(), z_u, e, s);
    }
  } else if (variant == FC_TUP) {
    Hierarchy &Hu = c.hier[FC_H_TUP_U], &Hp = c.hier[FC_H_TUP_P];
    if (nf) { k_face_hinv<TP><<<vgrid(nf), 256, 0, s>>>(nf, P.HinvT.p, w_t, P.tt.p); FS_LAUNCHED(); }
    sell_axpby<3, 3>(P.tC2.view(), P.tt.p, P.tu.p, 1.0, 1.0, w_u, s);        // t_u = w_u + C2^T H~^-T w_t
    amg_vcycle_t<TP>(Hu, P.tu.p, P.su.p, s);                                  // s_u = AMG^T(S1, t_u)
    sell_axpby<1, 3>(P.tQ1.view(), P.su.p, P.tp.p, -1.0, 1.0, w_p, s);       // t_p = w_p - Q1^T s_u
    if (nf) amg_vcycle<TP>(Hp, P.tp.p, z_p, s);                               // v_p = S~2^-T t_p
    sell_axpby<3, 1>(P.tQ2.view(), z_p, P.tu.p, 1.0, 0.0, (const TP *)nullptr, s);
    amg_vcycle_t<TP>(Hu, P.tu.p, z_u, s);                                     // AMG^T(S1, Q2^T v_p)
    axpbyz(z_u, P.su.p, z_u, 1.0, -1.0, nu, s);                               // v_u = s_u - ...
    if (nf) {                                                                 // v_t = H~^-T (C1^T v_u - w_t)
      EpiHinvUpdate<TP> e{z_t, P.tt.p, P.HinvT.p};
      sell_spmv<3, 3>(P.tC1.view(), z_u, e, s);
    }
  } else {
    Hierarchy &Hu = c.hier[FC_H_TPU_U], &Hp = c.hier[FC_H_TPU_P];
    if (nf) amg_vcycle<TP>(Hp, w_p, P.tp.p, s);                               // t_p = T^-T w_p
    if (nf) { k_face_hinv<TP><<<vgrid(nf), 256, 0, s>>>(nf, P.HinvT.p, w_t, P.tt.p); FS_LAUNCHED(); }
    sell_axpby<3, 3>(P.tC2.view(), P.tt.p, P.tu.p, 1.0, 1.0, w_u, s);
    sell_axpby<3, 1>(P.tQ2.view(), P.tp.p, P.tu.p, -1.0, 1.0, P.tu.p, s);  // t_u
    amg_vcycle_t<TP>(Hu, P.tu.p, z_u, s);                                     // v_u = AMG^T(S~, t_u)
    if (nf) {
      sell_axpby<1, 3>(P.tQ1.view(), z_u, P.sp.p, 1.0, 0.0, (const TP *)nullptr, s);
      amg_vcycle<TP>(Hp, P.sp.p, P.vp.p, s);
      axpbyz(z_p, P.tp.p, P.vp.p, 1.0, -1.0, nf, s);                          // v_p = t_p - T^-T Q1^T v_u
      EpiHinvUpdate<TP> e{z_t, P.tt.p, P.HinvT.p};                           // v_t = H~^-T (C1^T v_u - w_t)
      sell_spmv<3, 3>(P.tC1.view(), z_u, e, s);
    }
  }
}

template <typename TP>
PrecData<TP> &prec(fc_ctx &c);
template <>
PrecData<float> &prec<float>(fc_ctx &c) { return c.pf; }
template <>
PrecData<double> &prec<double>(fc_ctx &c) { return c.pd; }

template <typename TP>
TP *zbase(fc_ctx &c);
template <>
float *zbase<float>(fc_ctx &c) { return c.Zf.p; }
template <>
double *zbase<double>(fc_ctx &c) { return c.Zd.p; }

void ensure_krylov(fc_ctx &c, int maxit) {
  if (c.kcap >= maxit && c.kn == c.n && c.kprec == c.opt.precision) return;
  // invalidate first: a failed allocation below must not leave a workspace
  // that looks large enough
  c.kcap = 0;
  const int64_t n = c.n;
  c.V.alloc((size_t)(maxit + 1) * n);
  if (c.opt.precision == FC_MIXED) c.Zf.alloc((size_t)maxit * n);
  else c.Zd.alloc((size_t)maxit * n);
  c.Hm.alloc((size_t)(maxit + 1) * maxit);
  c.cs.alloc(maxit); c.sn.alloc(maxit); c.g.alloc(maxit + 1); c.y.alloc(maxit);
  c.hacc.alloc(maxit + 1); c.htmp.alloc(maxit + 1);
  c.partial.alloc((size_t)(maxit + 2) * (size_t)(kCgsSubGrid > kCgsDotGrid ? kCgsSubGrid : kCgsDotGrid));
  c.kcap = maxit;
  c.kn = n;
  c.kprec = c.opt.precision;
}

// Classical Gram-Schmidt applied twice against V_0..V_{m-1}:
//   h = V^T w; w -= V h; h' = V^T w; w -= V h'; h += h'
// with ||w||^2 before (w02) and after (w2) folded into the passes.
void cgs2(fc_ctx &c, int m, double *w) {
  NvtxRange nvtx("CGS2");
  const int64_t n = c.n;
  cudaStream_t s = c.s;
  const int nd = kCgsDotGrid, ns = kCgsSubGrid;
  const int fg = blocks_for((int64_t)(m + 1) * 32, 256, 1024);
  const size_t hsh = sizeof(double) * m;
  c.prof.start(PK_CGS, s);
  k_cgs_dot<<<nd, kCgsT, 0, s>>>(c.V.p, m, n, w, c.partial.p, 1);
  FS_LAUNCHED();
  k_cgs_final<<<fg, 256, 0, s>>>(c.partial.p, m, m + 1, nd, c.htmp.p, c.hacc.p, 0, c.w02.p);
  FS_LAUNCHED();
  k_cgs_sub<<<ns, kCgsT, hsh, s>>>(c.V.p, m, n, c.htmp.p, w, nullptr);
  FS_LAUNCHED();
  c.prof.stop(PK_CGS, s, (2.0 * m + 3.0) * n * sizeof(double));
  c.prof.start(PK_CGS, s);
  k_cgs_dot<<<nd, kCgsT, 0, s>>>(c.V.p, m, n, w, c.partial.p, 0);
  FS_LAUNCHED();
  k_cgs_final<<<fg, 256, 0, s>>>(c.partial.p, m, m, nd, c.htmp.p, c.hacc.p, 1, nullptr);
  FS_LAUNCHED();
  k_cgs_sub<<<ns, kCgsT, hsh, s>>>(c.V.p, m, n, c.htmp.p, w, c.partial.p);
  FS_LAUNCHED();
  k_cgs_final<<<1, 32, 0, s>>>(c.partial.p, 0, 1, ns, nullptr, nullptr, 0, c.w2.p);
  FS_LAUNCHED();
  c.prof.stop(PK_CGS, s, (2.0 * m + 3.0) * n * sizeof(double));
}

struct FgmresOut {
  int iters = 0;
  int status = FC_OK;
};

// one FGMRES cycle (no restart) on rhs r0 (device, double); dx written to x
template <typename TP, bool ADJ = false>
FgmresOut fgmres(fc_ctx &c, int variant, const double *rhs, double *x, double rtol, int maxit) {
  cudaStream_t s = c.s;
  const int64_t n = c.n;
  PrecData<TP> &P = prec<TP>(c);
  ensure_krylov(c, maxit);
  FgmresOut out;
  const double beta = std::sqrt(dot(rhs, rhs, n, s, c.red.p));
  if (!std::isfinite(beta)) { out.status = FC_NAN; return out; }
  if (beta == 0.0) {
    FS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    return out;
  }
  scale_to(c.V.p, rhs, 1.0 / beta, n, s);
  k_set_scalar<<<1, 1, 0, s>>>(c.g.p, beta);
  FS_LAUNCHED();
  TP *Z = zbase<TP>(c);
  int k = 0;
  for (int j = 0; j < maxit; j++) {
    double *vj = c.V.p + (int64_t)j * n;
    double *w = c.V.p + (int64_t)(j + 1) * n;
    TP *zj = Z + (int64_t)j * n;
    c.prof.start(PK_PREC, s);
    const TP *win;
    if constexpr (std::is_same<TP, double>::value) {
      win = vj;
    } else {
      cast(P.w.p, vj, n, s);
      win = P.w.p;
    }
    if constexpr (ADJ) apply_prec_t<TP>(c, P, variant, win, zj);
    else apply_prec<TP>(c, P, variant, win, zj);
    c.prof.stop(PK_PREC, s, 0.0);
    if constexpr (ADJ) jac_spmv_t<TP>(c, zj, w);
    else jac_spmv<TP>(c, zj, w);
    cgs2(c, j + 1, w);
    k_givens<<<1, 1, 0, s>>>(j, maxit + 1, c.hacc.p, c.w2.p, c.w02.p, beta, c.Hm.p, c.cs.p, c.sn.p, c.g.p, c.stat.p);
    FS_LAUNCHED();
    k_scale_by<<<vgrid(n), 256, 0, s>>>(w, n, c.stat.p + 3);
    FS_LAUNCHED();
    FS_CUDA(cudaMemcpyAsync(c.stat_host, c.stat.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    k = j + 1;
    const double est = c.stat_host[0];
    if (!std::isfinite(est)) { out.status = FC_NAN; break; }
    if (c.opt.verbose > 1) fprintf(stderr, "[fracsolve] it %d est %.3e\n", k, est);
    const bool breakdown = c.stat_host[3] == 0.0;
    if (est <= rtol) break;
    if (breakdown) { out.status = FC_BREAKDOWN; break; }
    if (k == maxit) out.status = FC_NOT_CONVERGED;
  }
  out.iters = k;
  c.kbasis = out.status == FC_BREAKDOWN ? k : k + 1;
  k_trisolve<<<1, 1, 0, s>>>(k, maxit + 1, c.Hm.p, c.g.p, c.y.p);
  FS_LAUNCHED();
  k_mcomb<TP><<<vgrid(n), 256, sizeof(double) * k, s>>>(Z, k, n, c.y.p, x);
  FS_LAUNCHED();
  return out;
}

template <typename TP, bool ADJ = false>
int solve_impl(fc_ctx &c, int variant, const double *b, double *x, double tol, int maxit, int *iters,
               double *relres) {
  NvtxRange nvtx(ADJ ? "fc_solve_adjoint" : "fc_solve");
  cudaStream_t s = c.s;
  const int64_t n = c.n;
  c.xk.ensure(n); c.rk.ensure(n);
  const double bn = std::sqrt(dot(b, b, n, s, c.red.p));
  if (!std::isfinite(bn)) return FC_NAN;
  int total = 0;
  int status = FC_OK;
  const double *rhs = b;
  double rr = 0.0;
  const int restarts = c.opt.precision == FC_MIXED ? std::max(0, (int)c.opt.max_restarts) : 0;
  FS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  if (bn == 0.0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return FC_OK;
  }
  for (int cycle = 0;; cycle++) {
    if (maxit - total <= 0) break;
    const double rn = cycle == 0 ? bn : std::sqrt(dot(rhs, rhs, n, s, c.red.p));
    const double rtol = tol * bn / rn;
    FgmresOut o = fgmres<TP, ADJ>(c, variant, rhs, c.xk.p, rtol, maxit - total);
    total += o.iters;
    axpby(x, c.xk.p, 1.0, 1.0, n, s);
    // true residual in double
    if constexpr (ADJ) jac_spmv_t<double>(c, x, c.rk.p);
    else jac_spmv<double>(c, x, c.rk.p);
    axpbyz(c.rk.p, b, c.rk.p, 1.0, -1.0, n, s);
    rr = std::sqrt(dot(c.rk.p, c.rk.p, n, s, c.red.p)) / bn;
    status = o.status;
    if (!std::isfinite(rr)) { status = FC_NAN; break; }
    if (rr <= tol) { status = FC_OK; break; }
    if (o.status == FC_NAN || cycle >= restarts || total >= maxit) {
      if (status == FC_OK) status = FC_NOT_CONVERGED;
      break;
    }
    rhs = c.rk.p;
  }
  if (iters) *iters = total;
  if (relres) *relres = rr;
  return status;
}

template <typename TP>
__global__ void k_transpose3(int64_t nf, const double *in, TP *out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 3; q++) out[f * 9 + q * 3 + r] = (TP)in[f * 9 + r * 3 + q];
}

template <typename TP>
void prepare_prec_t(fc_ctx &c, PrecData<TP> &P, const Bsr<double> &C1t, const Bsr<double> &C2t,
                    const Bsr<double> &Q1t, const Bsr<double> &Q2t) {
  cudaStream_t s = c.s;
  P.tC1 = to_sell<TP>(C1t.view(), s);
  P.tC2 = to_sell<TP>(C2t.view(), s);
  P.tQ1 = to_sell<TP>(Q1t.view(), s);
  P.tQ2 = to_sell<TP>(Q2t.view(), s);
  P.HinvT.alloc((size_t)c.nf * 9 > 0 ? (size_t)c.nf * 9 : 1);
  if (c.nf) {
    k_transpose3<TP><<<vgrid(c.nf), 256, 0, s>>>(c.nf, c.Hinv64.p, P.HinvT.p);
    FS_LAUNCHED();
  }
  P.ready_t = true;
}

// transposed blocks, transposed preconditioner data and transposed AMG
// cycles, built on the first adjoint call
void ensure_adjoint(fc_ctx &c) {
  if (c.have_adj) return;
  cudaStream_t s = c.s;
  Bsr<double> At = transpose(c.A.view(), s), C1t = transpose(c.C1.view(), s), Q1t = transpose(c.Q1.view(), s),
              C2t = transpose(c.C2.view(), s), Ht = transpose(c.H.view(), s), Q2t = transpose(c.Q2.view(), s),
              Tt = transpose(c.T.view(), s);
  c.tA = to_sell<double>(At.view(), s);
  c.tC1 = to_sell<double>(C1t.view(), s);
  c.tQ1 = to_sell<double>(Q1t.view(), s);
  c.tC2 = to_sell<double>(C2t.view(), s);
  c.tH = to_sell<double>(Ht.view(), s);
  c.tQ2 = to_sell<double>(Q2t.view(), s);
  c.tT = to_sell<double>(Tt.view(), s);
  if (c.opt.precision == FC_MIXED) prepare_prec_t<float>(c, c.pf, C1t, C2t, Q1t, Q2t);
  else prepare_prec_t<double>(c, c.pd, C1t, C2t, Q1t, Q2t);
  for (int h : {FC_H_TPU_U, FC_H_TUP_U})
    if (c.hier[h].built) amg_prepare_transpose(c.hier[h], c.opt.precision, s);
  FS_CUDA(cudaStreamSynchronize(s));
  c.have_adj = true;
}

}  // namespace

// ============================================================ residual without allocation
// Some callers cannot allocate device memory when they need a residual check:
// code that runs under a fixed device-memory budget reserved up front, code
// that must not let cudaFree synchronise the device in the middle of its
// stream work, or hosts that forbid further allocation once the solver is set
// up.  fc_residual_noalloc serves them: it keeps b - J x and its reduction
// partials in the file-scope arrays below (8 MiB + 4 KiB, held by every GPU
// that loads this library until the process exits) instead of caller or
// context buffers.
namespace {
constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;   // largest n accepted
constexpr int kNoAllocParts = 256;                   // reduction blocks
static __device__ __align__(256) double g_noalloc_r[kNoAllocMaxN];
static __device__ __align__(256) double g_noalloc_part[2 * kNoAllocParts + 2];

struct NoAllocScratch {
  double *r = nullptr;
  double *part = nullptr;
};
constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
NoAllocScratch g_noalloc_addr[kNoAllocDevices];

// device addresses of the scratch arrays on `device` (must be current);
// looked up once per device
int noalloc_scratch(int device, NoAllocScratch *out) {
  if (device < 0 || device >= kNoAllocDevices) return FC_BAD_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocScratch &a = g_noalloc_addr[device];
  if (!a.r) {
    void *r = nullptr, *p = nullptr;
    if (cudaGetSymbolAddress(&r, g_noalloc_r) != cudaSuccess ||
        cudaGetSymbolAddress(&p, g_noalloc_part) != cudaSuccess) {
      (void)cudaGetLastError();
      return FC_CUDA_ERROR;
    }
    a.r = static_cast<double *>(r);
    a.part = static_cast<double *>(p);
  }
  *out = a;
  return FC_OK;
}

// r = b - r (r holds J x on entry); per-block partial sums of r.r and b.b
__global__ void k_noalloc_resid(const double *__restrict__ b, double *r, int64_t n, double *part) {
  __shared__ double s_r[32], s_b[32];
  double ar = 0.0, ab = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const double v = bi - r[i];
    r[i] = v;
    ar += v * v;
    ab += bi * bi;
  }
  ar = warp_sum(ar);
  ab = warp_sum(ab);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s_r[wid] = ar; s_b[wid] = ab; }
  __syncthreads();
  if (wid == 0) {
    double x = lane < (int)(blockDim.x >> 5) ? s_r[lane] : 0.0;
    double y = lane < (int)(blockDim.x >> 5) ? s_b[lane] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    if (lane == 0) { part[blockIdx.x] = x; part[kNoAllocParts + blockIdx.x] = y; }
  }
}

// part[2P] = sum of the r.r partials, part[2P+1] = sum of the b.b partials
__global__ void k_noalloc_final(double *part) {
  const int lane = threadIdx.x;
  double x = 0.0, y = 0.0;
  for (int i = lane; i < kNoAllocParts; i += 32) { x += part[i]; y += part[kNoAllocParts + i]; }
  x = warp_sum(x);
  y = warp_sum(y);
  if (lane == 0) { part[2 * kNoAllocParts] = x; part[2 * kNoAllocParts + 1] = y; }
}
}  // namespace

// ============================================================ error plumbing
namespace {
int run(fc_ctx *c, const std::function<int()> &fn) {
  CacheScope scope(c ? &c->cache : nullptr);
  try {
    if (c) {
      c->err.clear();
      FS_CUDA(cudaSetDevice(c->device));
    }
    return fn();
  } catch (const Error &e) {
    if (c) c->err = e.what();
    (void)cudaGetLastError();
    return e.code;
  } catch (const std::bad_alloc &) {
    if (c) c->err = "host allocation failed";
    return FC_OOM;
  } catch (const std::exception &e) {
    if (c) c->err = e.what();
    return FC_INTERNAL;
  }
}
}  // namespace

extern "C" {

void fc_default_options(fc_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FC_FP64;
  o->variants = (1 << FC_TPU) | (1 << FC_TUP);
  o->theta0 = 0.08;
  o->theta_decay = 0.5;
  o->coarse_max = 200;
  o->coarse_max_p = 200;
  o->max_levels = 12;
  o->max_ratio = 0.8;
  o->power_steps = 15;
  o->omega_num = 4.0 / 3.0;
  o->cheb_degree = 2;
  o->cheb_hi = 1.1;
  o->cheb_lo = 0.1;
  o->amg_seed = 0;
  o->max_restarts = 3;
  o->verbose = 0;
  o->coarse_graphs = 1;
}

int fc_create(fc_ctx **out, const fc_options *opt, void *stream) {
  if (!out) return FC_BAD_ARG;
  *out = nullptr;
  std::unique_ptr<fc_ctx> c(new (std::nothrow) fc_ctx());
  if (!c) return FC_OOM;
  int rc = run(nullptr, [&]() {
    if (opt) c->opt = *opt;
    else fc_default_options(&c->opt);
    const fc_options &o = c->opt;
    FS_REQUIRE(o.precision == FC_FP64 || o.precision == FC_MIXED, FC_BAD_ARG, "precision");
    FS_REQUIRE((o.variants & 3) != 0, FC_BAD_ARG, "variants");
    FS_REQUIRE(o.cheb_degree >= 1 && o.cheb_degree <= 16, FC_BAD_ARG, "cheb_degree");
    FS_REQUIRE(o.coarse_max >= 1 && o.coarse_max_p >= 1 && o.max_levels >= 1, FC_BAD_ARG, "levels");
    FS_REQUIRE(o.cheb_hi > 0 && o.cheb_lo > 0 && o.cheb_lo < 1, FC_BAD_ARG, "chebyshev interval");
    FS_CUDA(cudaGetDevice(&c->device));
    c->s = (cudaStream_t)stream;
    FS_CUDA(cudaMallocHost(reinterpret_cast<void **>(&c->stat_host), 8 * sizeof(double)));
    c->stat.alloc(8);
    c->w2.alloc(1);
    c->w02.alloc(1);
    c->red.alloc(kRedBlocks + 1);
    return FC_OK;
  });
  if (rc == FC_OK) *out = c.release();
  return rc;
}

}  // extern "C"

namespace {
// The setup of Alg. 1 / Alg. 3 on device blocks J.  `staged` (optional)
// holds device copies of J's blocks that the context may keep as its own
// instead of copying them once more.
int setup_impl(fc_ctx *c, const fc_blocks *J, Bsr<double> *staged) {
    c->ready = false;
    const int nn = J->n_node, nf = J->n_face;
    FS_REQUIRE(nn > 0 && nf >= 0, FC_BAD_ARG, "n_node must be positive");
    check_bsr(J->A, nn, nn, 3, 3, "A", c->s);
    check_bsr(J->C1, nn, nf, 3, 3, "C1", c->s);
    check_bsr(J->Q1, nn, nf, 3, 1, "Q1", c->s);
    check_bsr(J->C2, nf, nn, 3, 3, "C2", c->s);
    check_bsr(J->H, nf, nf, 3, 3, "H", c->s);
    check_bsr(J->Q2, nf, nn, 1, 3, "Q2", c->s);
    check_bsr(J->T, nf, nf, 1, 1, "T", c->s);
    NvtxRange nvtx("fc_setup");
    cudaStream_t s = c->s;
    FS_REQUIRE(!c->geo.omega || c->geo_n == nf, FC_BAD_ARG,
               "geometric fixed-stress data was given for another face count; reset it with fc_set_geometric_fs");
    c->nn = nn; c->nf = nf;
    c->nu = 3LL * nn; c->nt = 3LL * nf; c->n = c->nu + c->nt + nf;
    fs::g_verbose = c->opt.verbose;
    PhaseTimer pt(c->opt.verbose > 0, s, "setup");
    auto up = [&](const fc_bsr &m, int k) {
      if (staged) return std::move(staged[k]);
      return upload_bsr(m.n_brows, m.n_bcols, m.br, m.bc, m.nnzb, m.d_row_ptr, m.d_col_idx, m.d_val, s);
    };
    c->A = up(J->A, 0); c->C1 = up(J->C1, 1); c->Q1 = up(J->Q1, 2); c->C2 = up(J->C2, 3);
    c->H = up(J->H, 4); c->Q2 = up(J->Q2, 5); c->T = up(J->T, 6);
    c->sA = to_sell<double>(c->A.view(), s); c->sC1 = to_sell<double>(c->C1.view(), s);
    c->sQ1 = to_sell<double>(c->Q1.view(), s); c->sC2 = to_sell<double>(c->C2.view(), s);
    c->sH = to_sell<double>(c->H.view(), s); c->sQ2 = to_sell<double>(c->Q2.view(), s);
    c->sT = to_sell<double>(c->T.view(), s);
    pt.mark("upload + sell");
    c->have_adj = false;
    for (auto &h : c->hier) h = Hierarchy();
    c->pf = PrecData<float>();
    c->pd = PrecData<double>();
    pt.mark("free old");
    build_hinv(c->H.view(), c->Hinv64, s);                                        // H~^-1 (Alg. 1, Alg. 3)
    c->S1 = build_s1(c->A.view(), c->C1.view(), c->C2.view(), c->Hinv64.p, s);   // S1 (Alg. 3)
    pt.mark("S1");
    const int prec = c->opt.precision;
    c->have[FC_TPU] = (c->opt.variants >> FC_TPU) & 1;
    c->have[FC_TUP] = (c->opt.variants >> FC_TUP) & 1;
    if (c->have[FC_TPU]) {
      c->St = build_stilde(c->S1.view(), c->Q1.view(), c->Q2.view(), c->T.view(), s);   // S~ (Alg. 1)
      amg_setup(c->hier[FC_H_TPU_U], copy_cast<double, double>(c->St.view(), s), 3, amg_params(c->opt, false), prec, s);
      if (nf) amg_setup(c->hier[FC_H_TPU_P], copy_cast<double, double>(c->T.view(), s), 1, amg_params(c->opt, true), prec, s);
    }
    if (c->have[FC_TUP]) {
      c->S2t = build_s2tilde(c->S1.view(), c->Q1.view(), c->Q2.view(), c->T.view(), c->SK, s, &c->geo);  // S~2 = T - FS (Alg. 3)
      pt.mark("S2tilde (fixed stress)");
      amg_setup(c->hier[FC_H_TUP_U], copy_cast<double, double>(c->S1.view(), s), 3, amg_params(c->opt, false), prec, s);
      if (nf) amg_setup(c->hier[FC_H_TUP_P], copy_cast<double, double>(c->S2t.view(), s), 1, amg_params(c->opt, true), prec, s);
    }
    c->hier[FC_H_TPU_U].prof = &c->prof;
    c->hier[FC_H_TUP_U].prof = &c->prof;
    pt.mark("hierarchies");
    if (prec == FC_MIXED) prepare_prec<float>(*c, c->pf);
    else prepare_prec<double>(*c, c->pd);
    c->xk.alloc(c->n); c->rk.alloc(c->n);
    pt.mark("prec data");
    FS_CUDA(cudaStreamSynchronize(s));
    c->ready = true;
    return FC_OK;
}

// device copy of a block whose arrays are in host memory
Bsr<double> stage_host_bsr(const fc_bsr &m, const char *name, cudaStream_t s) {
  FS_REQUIRE(m.n_brows >= 0 && m.n_bcols >= 0 && m.br > 0 && m.bc > 0 && m.nnzb >= 0 && m.d_row_ptr &&
                 (m.nnzb == 0 || (m.d_col_idx && m.d_val)),
             FC_BAD_ARG, std::string("block ") + name + " has inconsistent sizes or null pointers");
  Bsr<double> B;
  B.shape(m.n_brows, m.n_bcols, m.br, m.bc);
  B.nnzb = m.nnzb;
  B.rp.alloc((size_t)m.n_brows + 1);
  B.ci.alloc((size_t)std::max<int64_t>(m.nnzb, 1));
  B.val.alloc((size_t)std::max<int64_t>(m.nnzb, 1) * m.br * m.bc);
  FS_CUDA(cudaMemcpyAsync(B.rp.p, m.d_row_ptr, sizeof(int) * ((size_t)m.n_brows + 1), cudaMemcpyHostToDevice, s));
  if (m.nnzb) {
    FS_CUDA(cudaMemcpyAsync(B.ci.p, m.d_col_idx, sizeof(int) * (size_t)m.nnzb, cudaMemcpyHostToDevice, s));
    FS_CUDA(cudaMemcpyAsync(B.val.p, m.d_val, sizeof(double) * (size_t)m.nnzb * m.br * m.bc,
                            cudaMemcpyHostToDevice, s));
  }
  return B;
}
}  // namespace

extern "C" {

int fc_setup(fc_ctx *c, const fc_blocks *J) {
  if (!c || !J) return FC_BAD_ARG;
  return run(c, [&]() { return setup_impl(c, J, nullptr); });
}

int fc_setup_host(fc_ctx *c, const fc_blocks *J) {
  if (!c || !J) return FC_BAD_ARG;
  return run(c, [&]() {
    const fc_bsr *in[7] = {&J->A, &J->C1, &J->Q1, &J->C2, &J->H, &J->Q2, &J->T};
    const char *names[7] = {"A", "C1", "Q1", "C2", "H", "Q2", "T"};
    // sizes first: nothing is read from the host arrays of a block whose
    // dimensions do not fit the system
    const int nn = J->n_node, nf = J->n_face;
    FS_REQUIRE(nn > 0 && nf >= 0, FC_BAD_ARG, "n_node must be positive");
    const int dims[7][4] = {{nn, nn, 3, 3}, {nn, nf, 3, 3}, {nn, nf, 3, 1}, {nf, nn, 3, 3},
                            {nf, nf, 3, 3}, {nf, nn, 1, 3}, {nf, nf, 1, 1}};
    for (int k = 0; k < 7; k++)
      FS_REQUIRE(in[k]->n_brows == dims[k][0] && in[k]->n_bcols == dims[k][1] && in[k]->br == dims[k][2] &&
                     in[k]->bc == dims[k][3],
                 FC_BAD_ARG, std::string("block ") + names[k] + " has inconsistent sizes");
    Bsr<double> st[7];
    fc_blocks Jd = *J;
    fc_bsr *out[7] = {&Jd.A, &Jd.C1, &Jd.Q1, &Jd.C2, &Jd.H, &Jd.Q2, &Jd.T};
    for (int k = 0; k < 7; k++) {
      st[k] = stage_host_bsr(*in[k], names[k], c->s);
      out[k]->d_row_ptr = st[k].rp.p;
      out[k]->d_col_idx = st[k].ci.p;
      out[k]->d_val = st[k].val.p;
    }
    return setup_impl(c, &Jd, st);
  });
}

int fc_update(fc_ctx *c, const fc_blocks *J) {
  if (!c || !J) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_update needs a completed fc_setup");
    const int nn = c->nn, nf = c->nf;
    FS_REQUIRE(J->n_node == nn && J->n_face == nf, FC_BAD_ARG, "fc_update: sizes differ from the last fc_setup");
    check_bsr(J->A, nn, nn, 3, 3, "A", c->s);
    check_bsr(J->C1, nn, nf, 3, 3, "C1", c->s);
    check_bsr(J->Q1, nn, nf, 3, 1, "Q1", c->s);
    check_bsr(J->C2, nf, nn, 3, 3, "C2", c->s);
    check_bsr(J->H, nf, nf, 3, 3, "H", c->s);
    check_bsr(J->Q2, nf, nn, 1, 3, "Q2", c->s);
    check_bsr(J->T, nf, nf, 1, 1, "T", c->s);
    NvtxRange nvtx("fc_update");
    cudaStream_t s = c->s;
    fs::g_verbose = c->opt.verbose;
    PhaseTimer pt(c->opt.verbose > 0, s, "update");
    const fc_bsr *in[7] = {&J->A, &J->C1, &J->Q1, &J->C2, &J->H, &J->Q2, &J->T};
    Bsr<double> *own[7] = {&c->A, &c->C1, &c->Q1, &c->C2, &c->H, &c->Q2, &c->T};
    const char *names[7] = {"A", "C1", "Q1", "C2", "H", "Q2", "T"};
    bool changed[7];
    for (int k = 0; k < 7; k++) {
      BsrView<double> v;
      v.nbr = in[k]->n_brows; v.nbc = in[k]->n_bcols; v.br = in[k]->br; v.bc = in[k]->bc;
      v.nnzb = in[k]->nnzb; v.rp = in[k]->d_row_ptr; v.ci = in[k]->d_col_idx; v.val = in[k]->d_val;
      FS_REQUIRE(same_pattern(v, own[k]->view(), s), FC_BAD_ARG,
                 std::string("fc_update: the pattern of block ") + names[k] + " differs from the last fc_setup");
      const int64_t nv = v.nnzb * v.br * v.bc;
      changed[k] = !same_values(v.val, own[k]->val.p, nv, s);
    }
    c->ready = false;
    for (int k = 0; k < 7; k++) {
      const int64_t nv = own[k]->nnzb * own[k]->br * own[k]->bc;
      if (changed[k] && nv)
        FS_CUDA(cudaMemcpyAsync(own[k]->val.p, in[k]->d_val, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    }
    c->sA = to_sell<double>(c->A.view(), s); c->sC1 = to_sell<double>(c->C1.view(), s);
    c->sQ1 = to_sell<double>(c->Q1.view(), s); c->sC2 = to_sell<double>(c->C2.view(), s);
    c->sH = to_sell<double>(c->H.view(), s); c->sQ2 = to_sell<double>(c->Q2.view(), s);
    c->sT = to_sell<double>(c->T.view(), s);
    c->have_adj = false;
    pt.mark("pattern check + values");
    build_hinv(c->H.view(), c->Hinv64, s);
    Bsr<double> S1 = build_s1(c->A.view(), c->C1.view(), c->C2.view(), c->Hinv64.p, s);
    const bool s1_same = same_values(S1.val.p, c->S1.val.p, S1.nnzb * 9, s) && S1.nnzb == c->S1.nnzb;
    c->S1 = std::move(S1);
    pt.mark("S1");
    const int prec = c->opt.precision;
    if (c->have[FC_TPU]) {
      Bsr<double> St = build_stilde(c->S1.view(), c->Q1.view(), c->Q2.view(), c->T.view(), s);
      const bool st_same = St.nnzb == c->St.nnzb && same_values(St.val.p, c->St.val.p, St.nnzb * 9, s);
      c->St = std::move(St);
      if (!st_same) amg_refresh(c->hier[FC_H_TPU_U], copy_cast<double, double>(c->St.view(), s), prec, s);
      if (nf && changed[6]) amg_refresh(c->hier[FC_H_TPU_P], copy_cast<double, double>(c->T.view(), s), prec, s);
    }
    if (c->have[FC_TUP]) {
      Bsr<double> S2 = build_s2tilde(c->S1.view(), c->Q1.view(), c->Q2.view(), c->T.view(), c->SK, s, &c->geo);
      const bool s2_same = S2.nnzb == c->S2t.nnzb && same_values(S2.val.p, c->S2t.val.p, S2.nnzb, s);
      c->S2t = std::move(S2);
      if (!s1_same) amg_refresh(c->hier[FC_H_TUP_U], copy_cast<double, double>(c->S1.view(), s), prec, s);
      if (nf && !s2_same) amg_refresh(c->hier[FC_H_TUP_P], copy_cast<double, double>(c->S2t.view(), s), prec, s);
    }
    pt.mark("hierarchies");
    c->pf = PrecData<float>();
    c->pd = PrecData<double>();
    if (prec == FC_MIXED) prepare_prec<float>(*c, c->pf);
    else prepare_prec<double>(*c, c->pd);
    pt.mark("prec data");
    FS_CUDA(cudaStreamSynchronize(s));
    c->ready = true;
    return FC_OK;
  });
}

int fc_set_geometric_fs(fc_ctx *c, const double *omega, const double *kbar, double dt) {
  if (!c) return FC_BAD_ARG;
  return run(c, [&]() {
    if (!omega) {
      c->geo = GeoFs();
      c->geo_omega.release();
      c->geo_kbar.release();
      return FC_OK;
    }
    FS_REQUIRE(kbar && dt > 0.0, FC_BAD_ARG, "geometric fixed stress needs kbar and dt > 0");
    FS_REQUIRE(c->nf > 0, FC_NOT_SETUP, "geometric fixed stress: call fc_setup first (face count)");
    const int64_t nf = c->nf;
    c->geo_omega.alloc(nf);
    c->geo_kbar.alloc(nf);
    FS_CUDA(cudaMemcpyAsync(c->geo_omega.p, omega, sizeof(double) * nf, cudaMemcpyDeviceToDevice, c->s));
    FS_CUDA(cudaMemcpyAsync(c->geo_kbar.p, kbar, sizeof(double) * nf, cudaMemcpyDeviceToDevice, c->s));
    FS_CUDA(cudaStreamSynchronize(c->s));
    c->geo.omega = c->geo_omega.p;
    c->geo.kbar = c->geo_kbar.p;
    c->geo.dt = dt;
    c->geo_n = nf;
    return FC_OK;
  });
}

int fc_spmv(fc_ctx *c, const double *x, double *y) {
  if (!c || !x || !y) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    jac_spmv<double>(*c, x, y);
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

int fc_residual(fc_ctx *c, const double *b, const double *x, double *r, double *relres) {
  if (!c || !b || !x || !r) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    jac_spmv<double>(*c, x, r);
    axpbyz(r, b, r, 1.0, -1.0, c->n, c->s);
    const double rn = std::sqrt(dot(r, r, c->n, c->s, c->red.p));
    const double bn = std::sqrt(dot(b, b, c->n, c->s, c->red.p));
    if (relres) *relres = bn > 0 ? rn / bn : rn;
    return std::isfinite(rn) ? FC_OK : FC_NAN;
  });
}

int fc_apply_prec(fc_ctx *c, int variant, const double *w, double *v) {
  if (!c || !w || !v || !valid_variant(variant)) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready && built(*c, variant), FC_NOT_SETUP, "variant not built by fc_setup");
    if (c->opt.precision == FC_MIXED) {
      cast(c->pf.w.p, w, c->n, c->s);
      apply_prec<float>(*c, c->pf, variant, c->pf.w.p, c->pf.out.p);
      cast(v, c->pf.out.p, c->n, c->s);
    } else {
      apply_prec<double>(*c, c->pd, variant, w, v);
    }
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

int fc_solve(fc_ctx *c, int variant, const double *b, double *x, double tol, int maxit, int *iters,
             double *relres) {
  if (!c || !b || !x || !valid_variant(variant) || maxit < 1 || maxit > 4000 || !(tol > 0))
    return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready && built(*c, variant), FC_NOT_SETUP, "variant not built by fc_setup");
    int rc = c->opt.precision == FC_MIXED ? solve_impl<float>(*c, variant, b, x, tol, maxit, iters, relres)
                                          : solve_impl<double>(*c, variant, b, x, tol, maxit, iters, relres);
    FS_CUDA(cudaStreamSynchronize(c->s));
    return rc;
  });
}

int fc_solve_host(fc_ctx *c, int variant, const double *hb, double *hx, double tol, int maxit, int *iters,
                  double *relres) {
  if (!c || !hb || !hx) return FC_BAD_ARG;
  int rc = run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    c->bk.ensure(c->n);
    c->hx.ensure(c->n);
    FS_CUDA(cudaMemcpyAsync(c->bk.p, hb, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->s));
    return FC_OK;
  });
  if (rc != FC_OK) return rc;
  rc = fc_solve(c, variant, c->bk.p, c->hx.p, tol, maxit, iters, relres);
  int rc2 = run(c, [&]() {
    FS_CUDA(cudaMemcpyAsync(hx, c->hx.p, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->s));
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
  return rc != FC_OK ? rc : rc2;
}

int fc_spmv_adjoint(fc_ctx *c, const double *x, double *y) {
  if (!c || !x || !y) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    ensure_adjoint(*c);
    jac_spmv_t<double>(*c, x, y);
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

int fc_apply_prec_adjoint(fc_ctx *c, int variant, const double *w, double *v) {
  if (!c || !w || !v || !valid_variant(variant)) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready && built(*c, variant), FC_NOT_SETUP, "variant not built by fc_setup");
    ensure_adjoint(*c);
    if (c->opt.precision == FC_MIXED) {
      cast(c->pf.w.p, w, c->n, c->s);
      apply_prec_t<float>(*c, c->pf, variant, c->pf.w.p, c->pf.out.p);
      cast(v, c->pf.out.p, c->n, c->s);
    } else {
      apply_prec_t<double>(*c, c->pd, variant, w, v);
    }
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

int fc_solve_adjoint(fc_ctx *c, int variant, const double *g, double *lambda, double tol, int maxit, int *iters,
                     double *relres) {
  if (!c || !g || !lambda || !valid_variant(variant) || maxit < 1 || maxit > 4000 ||
      !(tol > 0))
    return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready && built(*c, variant), FC_NOT_SETUP, "variant not built by fc_setup");
    ensure_adjoint(*c);
    int rc = c->opt.precision == FC_MIXED
                 ? solve_impl<float, true>(*c, variant, g, lambda, tol, maxit, iters, relres)
                 : solve_impl<double, true>(*c, variant, g, lambda, tol, maxit, iters, relres);
    FS_CUDA(cudaStreamSynchronize(c->s));
    return rc;
  });
}

int fc_vcycle_adjoint(fc_ctx *c, int hier, const double *f, double *x) {
  if (!c || !f || !x || hier < 0 || hier > 3) return FC_BAD_ARG;
  return run(c, [&]() {
    Hierarchy &H = c->hier[hier];
    FS_REQUIRE(H.built, FC_NOT_SETUP, "hierarchy not built");
    amg_prepare_transpose(H, c->opt.precision, c->s);
    const int64_t n = (int64_t)H.lev[0].nb * H.B;
    if (c->opt.precision == FC_MIXED) {
      DBuf<float> f32(n), x32(n);
      cast(f32.p, f, n, c->s);
      amg_vcycle_t<float>(H, f32.p, x32.p, c->s);
      cast(x, x32.p, n, c->s);
    } else {
      amg_vcycle_t<double>(H, f, x, c->s);
    }
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

namespace {
// grad[f] = - sum over the derivative entries e of face f of
//   lambda_p[row_e] * val_e * x[col_e]   (x_p for T entries, x_u for Q2 entries)
// one warp per face, lane-strided sums reduced in a fixed tree
__global__ void k_check_face_ptr(int nf, const int64_t *fptr, int *flag) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    if ((f == 0 && fptr[0] != 0) || fptr[f + 1] < fptr[f]) atomicOr(flag, 1);
  }
}

// entries whose indices fall outside the system are skipped and flagged
__global__ void k_aperture_gradient(int nf, int nn, const int64_t *fptr, const int8_t *block, const int *row,
                                    const int *col, const int8_t *comp, const double *val, const double *x_u,
                                    const double *x_p, const double *lam_p, double *grad, int *flag) {
  const int lane = threadIdx.x & 31;
  for (int64_t f = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; f < nf;
       f += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int64_t e = fptr[f] + lane; e < fptr[f + 1]; e += 32) {
      const int b = block[e], r = row[e], cl = col[e], cp = comp[e];
      const bool ok = r >= 0 && r < nf &&
                      ((b == 0 && cl >= 0 && cl < nf) || (b == 1 && cl >= 0 && cl < nn && cp >= 0 && cp < 3));
      if (!ok) {
        atomicOr(flag, 2);
        continue;
      }
      const double xv = b == 0 ? x_p[cl] : x_u[3 * (int64_t)cl + cp];
      s += lam_p[r] * val[e] * xv;
    }
    s = warp_sum(s);
    if (lane == 0) grad[f] = -s;
  }
}
}  // namespace

int fc_aperture_gradient(fc_ctx *c, const int64_t *face_ptr, const int8_t *block, const int32_t *row,
                         const int32_t *col, const int8_t *comp, const double *val, const double *x,
                         const double *lambda, double *grad) {
  if (!c || !face_ptr || !x || !lambda || !grad) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    if (c->nf == 0) return FC_OK;
    FS_REQUIRE(block && row && col && comp && val, FC_BAD_ARG, "aperture gradient: null entry arrays");
    const double *x_u = x, *x_p = x + c->nu + c->nt, *lam_p = lambda + c->nu + c->nt;
    DBuf<int> flag(1);
    FS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), c->s));
    k_check_face_ptr<<<blocks_for(c->nf, 256, kSMs * 8), 256, 0, c->s>>>(c->nf, face_ptr, flag.p);
    FS_LAUNCHED();
    int h = 0;
    FS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    FS_CUDA(cudaStreamSynchronize(c->s));
    FS_REQUIRE(!h, FC_BAD_ARG, "aperture gradient: face_ptr must start at 0 and not decrease");
    k_aperture_gradient<<<blocks_for((int64_t)c->nf * 32, 256, kSMs * 16), 256, 0, c->s>>>(
        c->nf, c->nn, face_ptr, block, row, col, comp, val, x_u, x_p, lam_p, grad, flag.p);
    FS_LAUNCHED();
    FS_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    FS_CUDA(cudaStreamSynchronize(c->s));
    FS_REQUIRE(!h, FC_BAD_ARG, "aperture gradient: an entry's row, column or component is out of range");
    return FC_OK;
  });
}

int fc_num_levels(fc_ctx *c, int hier, int *levels) {
  if (!c || !levels || hier < 0 || hier > 3) return FC_BAD_ARG;
  *levels = c->hier[hier].built ? c->hier[hier].levels() : 0;
  return FC_OK;
}

int fc_get_bsr(fc_ctx *c, int kind, int hier, int level, int32_t *nbr, int32_t *nbc, int32_t *br, int32_t *bc,
               int64_t *nnzb, int32_t *hrp, int32_t *hci, double *hval) {
  if (!c) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    const Bsr<double> *m = nullptr;
    if (kind == FC_M_S1) m = &c->S1;
    else if (kind == FC_M_STILDE) m = &c->St;
    else if (kind == FC_M_S2TILDE) m = &c->S2t;
    else if (kind == FC_M_LEVEL || kind == FC_M_PROLONG) {
      FS_REQUIRE(hier >= 0 && hier < 4 && c->hier[hier].built, FC_BAD_ARG, "hierarchy not built");
      FS_REQUIRE(level >= 0 && level < c->hier[hier].levels(), FC_BAD_ARG, "level out of range");
      const LevelSetup &L = c->hier[hier].lev[level];
      m = kind == FC_M_LEVEL ? &L.S : &L.P;
    } else {
      throw Error(FC_BAD_ARG, "unknown matrix kind");
    }
    if (nbr) *nbr = m->nbr;
    if (nbc) *nbc = m->nbc;
    if (br) *br = m->br;
    if (bc) *bc = m->bc;
    if (nnzb) *nnzb = m->nnzb;
    if (hrp || hci || hval) {
      std::vector<int> rp, ci;
      std::vector<double> val;
      download_bsr(m->view(), rp, ci, val, c->s);
      if (hrp) std::memcpy(hrp, rp.data(), sizeof(int) * rp.size());
      if (hci && !ci.empty()) std::memcpy(hci, ci.data(), sizeof(int) * ci.size());
      if (hval && !val.empty()) std::memcpy(hval, val.data(), sizeof(double) * val.size());
    }
    return FC_OK;
  });
}

int fc_get_aggregates(fc_ctx *c, int hier, int level, int32_t *hagg, double *hlam) {
  if (!c || hier < 0 || hier > 3) return FC_BAD_ARG;
  return run(c, [&]() {
    Hierarchy &H = c->hier[hier];
    FS_REQUIRE(H.built && level >= 0 && level < H.levels(), FC_BAD_ARG, "level out of range");
    const LevelSetup &L = H.lev[level];
    if (hlam) *hlam = L.lam;
    if (hagg) {
      if (L.agg.p) {
        FS_CUDA(cudaMemcpyAsync(hagg, L.agg.p, sizeof(int) * L.nb, cudaMemcpyDeviceToHost, c->s));
      } else {
        for (int i = 0; i < L.nb; i++) hagg[i] = -1;
      }
      FS_CUDA(cudaStreamSynchronize(c->s));
    }
    return FC_OK;
  });
}

int fc_vcycle(fc_ctx *c, int hier, const double *f, double *x) {
  if (!c || !f || !x || hier < 0 || hier > 3) return FC_BAD_ARG;
  return run(c, [&]() {
    Hierarchy &H = c->hier[hier];
    FS_REQUIRE(H.built, FC_NOT_SETUP, "hierarchy not built");
    const int64_t n = (int64_t)H.lev[0].nb * H.B;
    if (c->opt.precision == FC_MIXED) {
      DBuf<float> f32(n), x32(n);
      cast(f32.p, f, n, c->s);
      amg_vcycle<float>(H, f32.p, x32.p, c->s);
      cast(x, x32.p, n, c->s);
      FS_CUDA(cudaStreamSynchronize(c->s));
    } else {
      amg_vcycle<double>(H, f, x, c->s);
      FS_CUDA(cudaStreamSynchronize(c->s));
    }
    return FC_OK;
  });
}

int fc_get_fixed_stress(fc_ctx *c, double *hsk) {
  if (!c || !hsk) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready && c->have[FC_TUP], FC_NOT_SETUP, "t-u-p not built");
    if (c->nf)
      FS_CUDA(cudaMemcpyAsync(hsk, c->SK.p, sizeof(double) * c->nf, cudaMemcpyDeviceToHost, c->s));
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

int fc_profile(fc_ctx *c, int enable) {
  if (!c) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_CUDA(cudaStreamSynchronize(c->s));
    c->prof.reset();
    c->prof.on = enable != 0;
    return FC_OK;
  });
}

int fc_kernel_stats(fc_ctx *c, int kernel, int64_t *launches, double *total_ms, double *bytes) {
  if (!c || kernel < 0 || kernel >= PK_N) return FC_BAD_ARG;
  return run(c, [&]() {
    c->prof.stats(kernel, launches, total_ms, bytes);
    return FC_OK;
  });
}

unsigned long long fc_launch_count(void) { return fs::launch_count(); }

int fc_krylov_basis(fc_ctx *c, int *nvec, double *d_V) {
  if (!c || !nvec) return FC_BAD_ARG;
  return run(c, [&]() {
    *nvec = c->kbasis;
    if (d_V && c->kbasis)
      FS_CUDA(cudaMemcpyAsync(d_V, c->V.p, sizeof(double) * (size_t)c->kbasis * c->n, cudaMemcpyDeviceToDevice,
                              c->s));
    FS_CUDA(cudaStreamSynchronize(c->s));
    return FC_OK;
  });
}

int fc_residual_noalloc(fc_ctx *c, const double *b, const double *x, double *relres) {
  if (!c || !b || !x || !relres) return FC_BAD_ARG;
  return run(c, [&]() {
    FS_REQUIRE(c->ready, FC_NOT_SETUP, "fc_setup has not completed");
    FS_REQUIRE(c->n <= kNoAllocMaxN, FC_BAD_ARG,
               "fc_residual_noalloc: n = " + std::to_string(c->n) +
                   " exceeds the 1048576-entry scratch; use fc_residual");
    NoAllocScratch sc;
    const int rc = noalloc_scratch(c->device, &sc);
    FS_REQUIRE(rc == FC_OK, rc, "cudaGetSymbolAddress of the residual scratch failed");
    cudaStream_t s = c->s;
    // J x into the scratch by the solver's own product (a double direction
    // needs no widening buffer, so nothing is allocated)
    jac_spmv<double>(*c, x, sc.r);
    k_noalloc_resid<<<kNoAllocParts, 256, 0, s>>>(b, sc.r, c->n, sc.part);
    FS_LAUNCHED();
    k_noalloc_final<<<1, 32, 0, s>>>(sc.part);
    FS_LAUNCHED();
    FS_CUDA(cudaMemcpyAsync(c->stat_host + 4, sc.part + 2 * kNoAllocParts, 2 * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    FS_CUDA(cudaStreamSynchronize(s));
    const double rn = std::sqrt(c->stat_host[4]), bn = std::sqrt(c->stat_host[5]);
    *relres = bn > 0 ? rn / bn : rn;
    return std::isfinite(rn) ? FC_OK : FC_NAN;
  });
}

void fc_destroy(fc_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->s);
  delete c;
}

const char *fc_strerror(int st) {
  switch (st) {
    case FC_OK: return "ok";
    case FC_NOT_CONVERGED: return "not converged within maxit";
    case FC_BREAKDOWN: return "Krylov breakdown before reaching the tolerance";
    case FC_SINGULAR_BLOCK: return "singular block";
    case FC_NAN: return "NaN or Inf encountered";
    case FC_BAD_ARG: return "invalid argument";
    case FC_CUDA_ERROR: return "CUDA runtime error";
    case FC_OOM: return "out of device memory";
    case FC_INTERNAL: return "internal capacity limit reached";
    case FC_NOT_SETUP: return "setup has not built what the call needs";
    default: return "unknown status";
  }
}

const char *fc_last_error(fc_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
