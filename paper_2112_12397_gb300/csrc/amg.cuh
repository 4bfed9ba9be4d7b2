// Smoothed-aggregation AMG: hierarchy construction on the device (double)
// and the V(1,1)-cycle with a Chebyshev smoother (float or double).
#pragma once

#include <memory>

#include "common.cuh"
#include "sell.cuh"

namespace fs {

struct AmgParams {
  double theta0 = 0.08, theta_decay = 0.5;
  int coarse_max = 1000, max_levels = 12;
  double max_ratio = 0.8;
  int power_steps = 15;
  double omega_num = 4.0 / 3.0;
  int cheb_degree = 2;
  double cheb_hi = 1.1, cheb_lo = 0.1;
  uint64_t seed = 0;
  int verbose = 0;
  bool graphs = true;   // replay the coarse levels of the cycle as a CUDA graph
};

// Per-level data built in double precision.
struct LevelSetup {
  int B = 3, nb = 0;
  Bsr<double> S;        // level operator
  Bsr<double> P, R;     // prolongator (nb x nc blocks) and R = P^T (not on the coarsest)
  DBuf<double> Dinv;    // nb * B * B inverse diagonal blocks
  DBuf<int> agg;        // aggregate of each block row (-1: none)
  DBuf<int> asize;      // size of each aggregate
  int nc = 0;           // number of aggregates (coarse block rows)
  Bsr<double> SP;       // S P, kept for numeric rebuilds (FP64 mode)
  Bsr<float> SPf;       // S P in float (mixed mode: the Galerkin products run in float)
  double lam = 0.0;     // power estimate of the largest eigenvalue of D^-1 S
  // sliced-ELL operator and D^-1 in the cycle precision, built during setup
  // (the power iteration runs on them) and handed to the cycle
  Sell<float> Ssf;
  Sell<double> Ssd;
  Bsr<float> Sbf;                // float BSR copy of a long-row level (power steps, then the cycle)
  DBuf<float> Dinvf;
};

// Level operator as seen by the cycle: sliced ELL (one thread per row) for
// short rows, BSR with a lane group per row for long rows (coarse levels).
template <typename TP>
struct LevelOp {
  bool sell = true;
  bool chunk = false;            // long rows in chunked BSR
  ChunkView<TP> kv;
  SellView<TP> sv;
  BsrView<TP> bv;
  int64_t nnzb = 0;
  int nbr = 0;
};

// Per-level data of the cycle in precision TP.
template <typename TP>
struct LevelCycle {
  LevelOp<TP> op, opT;           // S and S^T as used by the cycle
  Bsr<TP> St_own;                // S^T in BSR form for long-row levels
  BsrView<TP> S, P, R;
  const TP *Dinv = nullptr;
  Bsr<TP> S_own, P_own, R_own;   // used when TP differs from double
  Sell<TP> Ss, Ps;               // sliced-ELL copies of S and P used by the cycle
  Sell<TP> SsT;                  // S^T for the transposed cycle (adjoint solves)
  Jag<TP> PSP;                   // [P | S P] for the fused prolongation and first post-smoothing step
  Chunked<TP> Sk, Rk;            // chunked copies of a long-row S and of R
  DBuf<TP> DinvT;                // transposed diagonal blocks
  DBuf<TP> Dinv_own;
  DBuf<TP> f, x, xa, d, r;       // right-hand side, iterate (two buffers), direction, residual
  double theta = 0, delta = 0, sigma = 0;
};

// An instantiated CUDA graph (move-only) and the kernel launches it replays.
struct GraphExec {
  cudaGraphExec_t g = nullptr;
  unsigned long long kernels = 0;
  GraphExec() = default;
  GraphExec(const GraphExec &) = delete;
  GraphExec &operator=(const GraphExec &) = delete;
  GraphExec(GraphExec &&o) noexcept : g(o.g), kernels(o.kernels) { o.g = nullptr; }
  GraphExec &operator=(GraphExec &&o) noexcept {
    if (this != &o) {
      reset();
      g = o.g;
      kernels = o.kernels;
      o.g = nullptr;
    }
    return *this;
  }
  ~GraphExec() { reset(); }
  void reset() {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
    kernels = 0;
  }
};

struct Hierarchy {
  int B = 3;
  bool built = false;
  AmgParams prm;
  std::vector<LevelSetup> lev;
  // coarsest level: explicit inverse in double, n_c x n_c row-major
  DBuf<double> cinv;
  int nc_scalar = 0;
  std::vector<LevelCycle<float>> cf;
  std::vector<LevelCycle<double>> cd;
  Profiler *prof = nullptr;      // times the level-0 smoother steps when set
  bool have_t = false;           // transposed cycle data built
  DBuf<double> cinvT;            // transposed coarsest inverse
  // levels 1 .. of the cycle as one graph: [double precision][transposed];
  // its buffers (level-1 f and x and below) are fixed for the hierarchy
  bool graphs = true;
  GraphExec coarse[2][2];
  // the whole cycle of a small scalar hierarchy as one graph, on its level-0
  // buffers: [double precision]
  GraphExec whole[2];
  int levels() const { return (int)lev.size(); }
};

// Build the hierarchy of S0 (block size B, square, sorted rows).  Takes
// ownership of S0.  precision: FC_FP64 or FC_MIXED (casts the cycle data).
void amg_setup(Hierarchy &H, Bsr<double> &&S0, int B, const AmgParams &prm, int precision,
               cudaStream_t s);

// Numeric rebuild of a built hierarchy for new values of its level-0
// operator with the same pattern (aggregates and all patterns kept).
// Takes ownership of S0; FC_BAD_ARG if the pattern differs.
void amg_refresh(Hierarchy &H, Bsr<double> &&S0, int precision, cudaStream_t s);

// x = V-cycle(f) with zero initial guess; f and x have nb(0) * B entries.
template <typename TP>
void amg_vcycle(Hierarchy &H, const TP *f, TP *x, cudaStream_t s);

// Data of the transposed cycle: S_l^T, transposed diagonal blocks and
// coarsest inverse (P and R are shared with the forward cycle).
void amg_prepare_transpose(Hierarchy &H, int precision, cudaStream_t s);

// x = B^T f: the transpose of the V-cycle operator, i.e. the same cycle on
// the transposed level operators.
template <typename TP>
void amg_vcycle_t(Hierarchy &H, const TP *f, TP *x, cudaStream_t s);

}  // namespace fs
