// Seeded fractured-cube instances assembled on the device: the mesh with its
// nodes split across the fracture faces, the material field, contact states
// and slip data, the seven blocks of the Jacobian (Eq. JacSys, Eq. block_def)
// and the right-hand side.
//
// Every sparsity pattern is enumerated directly from the mesh (no coordinate
// list, no sort): a row knows its candidate columns from the grid (the 27
// grid neighbours of a node, the 12 cell faces around a node, the 8 corners
// of a face, the faces on the 4 edges of a face), visits them in increasing
// column order, and is written by a count pass, a scan and a fill pass.
// Values follow the paper's definitions with the synthetic readings listed
// below; the entries agree with the host generator of the test suite up to
// the rounding of sums taken in another order.
//
// Readings where the paper is silent (shared with the host generator, which
// is the reference the parity tests use):
//  * units MPa, m, s; E = E0 exp(sigma Z) per cell (E0 = 10 GPa), nu = 0.25;
//    trilinear hexahedra, 2x2x2 Gauss; rollers on the six outer faces;
//  * counter-based draws r(seed, stream, i) (SplitMix64); streams 1 E, 2
//    state, 3 t_N, 4 slip angle, 5 |dg_T|, 6 aperture, 7 p^l, 8 b, 9
//    rectangles; Z by Box-Muller from draws 2i and 2i+1;
//  * stabilisation Ups = beta h^3 diag(1/M, 1/G, 1/G) on the edges between
//    coplanar faces (M, G from the mean E of the four cells), j_p its normal
//    part scaled by 1/dt (Sec. 2.2); k = Ebar_f / (k_scale h);
//  * TPFA with one-sided transmissibility 2 C_f / mu, C_f = C_f0 + a^3 / 12
//    (Eq. cond_def), series average over every pair of faces sharing an edge;
//    p = 0 on the outer edges of the corner faces of each fracture that no
//    other face touches;
//  * F_u: the derivative of the TPFA flux through the open faces' apertures,
//    g = mean normal jump of the face's copies (Eq. Q2vsQ1).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

namespace fs {
namespace {

constexpr double kE0 = 1.0e4;         // MPa (10 GPa)
constexpr double kNu = 0.25;
constexpr double kMu = 1.0e-9;        // MPa s (1e-3 Pa s)
constexpr double kDt = 0.5;           // s
constexpr double kCf0 = 9.87e-15;     // m^3, conductivity of closed faces
constexpr int kMaxNbr = 12;           // faces sharing an edge with a face

enum { S_E = 1, S_STATE = 2, S_TN = 3, S_PHI = 4, S_DG = 5, S_APER = 6, S_PL = 7, S_RHS = 8, S_RECT = 9 };

struct Fracture {
  int a, m, p0, q0, p1, q1;
};

__host__ __device__ inline double gauss_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  const double u1 = 1.0 - sm64_uniform(seed, stream, 2 * i);   // (0, 1]
  const double u2 = sm64_uniform(seed, stream, 2 * i + 1);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

struct Geo {
  int N, N1;
  double h;
  __device__ int64_t fidx(int a, int m, int p, int q) const {
    return (((int64_t)a * N1 + m) * N + q) * N + p;
  }
  __device__ int64_t cell(int x, int y, int z) const { return x + (int64_t)N * (y + (int64_t)N * z); }
};

// ------------------------------------------------------------------ faces
// owner of each interior cell face (lowest fracture index covering it)
__global__ void k_face_flags(Geo g, const Fracture *fr, int n_fr, int *flag) {
  const int64_t total = (int64_t)3 * g.N1 * g.N * g.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(k % g.N), q = (int)((k / g.N) % g.N);
    const int m = (int)((k / ((int64_t)g.N * g.N)) % g.N1), a = (int)(k / ((int64_t)g.N * g.N * g.N1));
    int hit = 0;
    for (int r = 0; r < n_fr && !hit; r++) {
      const Fracture f = fr[r];
      hit = f.a == a && f.m == m && p >= f.p0 && p <= f.p1 && q >= f.q0 && q <= f.q1;
    }
    flag[k] = hit;
  }
}

// face ids in (a, m, q, p) order and their geometry
__global__ void k_face_ids(Geo g, const int *flag, const int *pre, int *fmap, int *geom) {
  const int64_t total = (int64_t)3 * g.N1 * g.N * g.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[k]) {
      fmap[k] = -1;
      continue;
    }
    const int f = pre[k];
    fmap[k] = f;
    geom[4 * f + 0] = (int)(k / ((int64_t)g.N * g.N * g.N1));
    geom[4 * f + 1] = (int)((k / ((int64_t)g.N * g.N)) % g.N1);
    geom[4 * f + 2] = (int)(k % g.N);
    geom[4 * f + 3] = (int)((k / g.N) % g.N);
  }
}

// ------------------------------------------------------------------ node split
// Components of the (up to) 8 cells around grid node (I, J, K): cells e and
// e | 2^d are joined when the cell face between them is not fractured.  Cell
// e sits at (I-1, J-1, K-1) + bits(e), so cell ids grow with e and a
// component's smallest cell is its smallest e.  label[e] = smallest e of its
// component (-1: no cell).
__device__ int node_components(const Geo &g, const int *fmap, int I, int J, int K, int label[8]) {
  const int G[3] = {I, J, K};
  for (int e = 0; e < 8; e++) {
    const int c[3] = {I - 1 + (e & 1), J - 1 + ((e >> 1) & 1), K - 1 + ((e >> 2) & 1)};
    const bool ok = c[0] >= 0 && c[0] < g.N && c[1] >= 0 && c[1] < g.N && c[2] >= 0 && c[2] < g.N;
    label[e] = ok ? e : -1;
  }
  unsigned joined = 0;   // bit (e * 3 + d): edge e -- e | 2^d open
  for (int e = 0; e < 8; e++)
    for (int d = 0; d < 3; d++) {
      if ((e >> d) & 1) continue;
      const int e2 = e | (1 << d);
      if (label[e] < 0 || label[e2] < 0) continue;
      const int c[3] = {I - 1 + (e & 1), J - 1 + ((e >> 1) & 1), K - 1 + ((e >> 2) & 1)};
      const int p = c[(d + 1) % 3], q = c[(d + 2) % 3];
      if (fmap[g.fidx(d, G[d], p, q)] < 0) joined |= 1u << (e * 3 + d);
    }
  // min-label propagation over the cube's 12 edges (diameter 3)
  for (int it = 0; it < 4; it++)
    for (int e = 0; e < 8; e++)
      for (int d = 0; d < 3; d++) {
        if (!((joined >> (e * 3 + d)) & 1)) continue;
        const int e2 = e | (1 << d);
        const int l = min(label[e], label[e2]);
        label[e] = label[e2] = l;
      }
  int n = 0;
  for (int e = 0; e < 8; e++) n += label[e] == e;
  return n;
}

__global__ void k_node_count(Geo g, const int *fmap, int *cnt) {
  const int64_t total = (int64_t)g.N1 * g.N1 * g.N1;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < total; n += (int64_t)gridDim.x * blockDim.x) {
    int label[8];
    cnt[n] = node_components(g, fmap, (int)(n % g.N1), (int)((n / g.N1) % g.N1), (int)(n / ((int64_t)g.N1 * g.N1)),
                             label);
  }
}

// copies of each node in the order of their smallest cell: grid id, cell
// mask and the copy of every (cell, corner)
__global__ void k_node_split(Geo g, const int *fmap, const int *first, int *copy_grid, uint8_t *copy_mask,
                             int *cellnode) {
  const int64_t total = (int64_t)g.N1 * g.N1 * g.N1;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < total; n += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(n % g.N1), J = (int)((n / g.N1) % g.N1), K = (int)(n / ((int64_t)g.N1 * g.N1));
    int label[8];
    node_components(g, fmap, I, J, K, label);
    int rank[8];
    int r = 0;
    for (int e = 0; e < 8; e++)
      if (label[e] == e) rank[e] = r++;
    const int base = first[n];
    for (int e = 0; e < 8; e++) {
      if (label[e] < 0) continue;
      const int cid = base + rank[label[e]];
      if (label[e] == e) {
        uint8_t mk = 0;
        for (int e2 = 0; e2 < 8; e2++)
          if (label[e2] == e) mk |= (uint8_t)(1u << e2);
        copy_grid[cid] = (int)n;
        copy_mask[cid] = mk;
      }
      const int64_t c = g.cell(I - 1 + (e & 1), J - 1 + ((e >> 1) & 1), K - 1 + ((e >> 2) & 1));
      cellnode[8 * c + (7 - e)] = cid;   // the node is corner 7 - e of cell e
    }
  }
}

__global__ void k_material(Geo g, uint64_t seed, double sigma, double *E) {
  const int64_t total = (int64_t)g.N * g.N * g.N;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x)
    E[c] = kE0 * exp(sigma * gauss_draw(seed, S_E, (uint64_t)c));
}

// rollers: the normal component of every copy on an outer face of the cube
__global__ void k_dirichlet(Geo g, const int *copy_grid, int nn, int8_t *dir) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    const int gid = copy_grid[i];
    const int G[3] = {gid % g.N1, (gid / g.N1) % g.N1, gid / (g.N1 * g.N1)};
    for (int d = 0; d < 3; d++) dir[3 * i + d] = (G[d] == 0 || G[d] == g.N) ? 1 : 0;
  }
}

// ------------------------------------------------------------------ A
// Row i (a copy of grid node G): the copies sharing a cell with it are
// copies of the 27 grid neighbours, visited in grid order (copy ids follow
// grid ids), each copy in id order.  Shared cells are found from the two
// cell masks: cell e of G is cell e - (H - G) of H when that offset is 0/1.
struct ARow {
  __device__ static int shared(int e_mask_i, int mask_j, int dx, int dy, int dz, int out_i[8], int out_j[8]) {
    int n = 0;
    for (int e = 0; e < 8; e++) {
      if (!((e_mask_i >> e) & 1)) continue;
      const int bx = (e & 1) - dx, by = ((e >> 1) & 1) - dy, bz = ((e >> 2) & 1) - dz;
      if (bx < 0 || bx > 1 || by < 0 || by > 1 || bz < 0 || bz > 1) continue;
      const int eh = bx + 2 * by + 4 * bz;
      if ((mask_j >> eh) & 1) {
        out_i[n] = e;
        out_j[n] = eh;
        n++;
      }
    }
    return n;
  }
};

template <bool FILL>
__global__ void k_assemble_A(Geo g, int nn, const int *copy_grid, const uint8_t *copy_mask, const int *first,
                             const double *E, const double *__restrict__ Khat, const int8_t *dir, int *cnt,
                             const int *rp, int *ci, double *val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    const int gid = copy_grid[i];
    const int I = gid % g.N1, J = (gid / g.N1) % g.N1, K = gid / (g.N1 * g.N1);
    const int mi = copy_mask[i];
    int k = FILL ? rp[i] : 0;
    for (int dz = -1; dz <= 1; dz++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
          const int x = I + dx, y = J + dy, z = K + dz;
          if (x < 0 || x > g.N || y < 0 || y > g.N || z < 0 || z > g.N) continue;
          const int h = x + g.N1 * (y + g.N1 * z);
          for (int j = first[h]; j < first[h + 1]; j++) {
            int ei[8], ej[8];
            const int ns = ARow::shared(mi, copy_mask[j], dx, dy, dz, ei, ej);
            if (!ns) continue;
            if (FILL) {
              double b[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
              for (int t = 0; t < ns; t++) {   // shared cells in increasing id
                const int e = ei[t];
                const double s = E[g.cell(I - 1 + (e & 1), J - 1 + ((e >> 1) & 1), K - 1 + ((e >> 2) & 1))] * g.h;
                const int li = 7 - e, lj = 7 - ej[t];
                for (int r = 0; r < 3; r++)
                  for (int c = 0; c < 3; c++) b[3 * r + c] += s * Khat[(3 * li + r) * 24 + 3 * lj + c];
              }
              // symmetric elimination of the rollers (the diagonal stays)
              for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++)
                  if ((dir[3 * i + r] || dir[3 * j + c]) && !(i == j && r == c)) b[3 * r + c] = 0.0;
              ci[k] = j;
              for (int t = 0; t < 9; t++) val[(int64_t)k * 9 + t] = b[t];
            }
            k++;
          }
        }
    if (!FILL) cnt[i] = k;
  }
}

// ------------------------------------------------------------------ per-face data
struct FaceData {
  int8_t *state;
  double *aper, *pl, *ebar, *ups, *tn, *g1, *g2, *dg;
  int *copies;      // 8 per face: minus corners 0..3, plus corners 0..3
  int64_t *cells;   // 2 per face: minus, plus cell
};

__global__ void k_face_data(Geo g, int nf, const int *geom, const int *cellnode, const double *E, uint64_t seed,
                            double p_stick, double p_slip, double aper_sigma, const double *aper_in,
                            double pl_scale, FaceData F) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int a = geom[4 * f], m = geom[4 * f + 1], p = geom[4 * f + 2], q = geom[4 * f + 3];
    const double U = sm64_uniform(seed, S_STATE, f);
    F.state[f] = U < p_stick ? 0 : (U < p_stick + p_slip ? 1 : 2);
    const double ap = aper_in ? aper_in[f] : 1e-3 * exp(aper_sigma * gauss_draw(seed, S_APER, f));
    F.aper[f] = ap;
    F.pl[f] = pl_scale * sm64_uniform(seed, S_PL, f);
    F.tn[f] = -(5.0 + 10.0 * sm64_uniform(seed, S_TN, f));
    const double phi = 2.0 * M_PI * sm64_uniform(seed, S_PHI, f);
    F.g1[f] = cos(phi);
    F.g2[f] = sin(phi);
    F.dg[f] = 1e-4 * exp(0.5 * gauss_draw(seed, S_DG, f));
    for (int s = 0; s < 2; s++) {
      int c[3];
      c[a] = m - 1 + s;
      c[(a + 1) % 3] = p;
      c[(a + 2) % 3] = q;
      const int64_t cid = g.cell(c[0], c[1], c[2]);
      F.cells[2 * f + s] = cid;
      for (int k = 0; k < 4; k++) {
        int off[3];
        off[a] = 1 - s;                 // the face is the far side of the minus cell
        off[(a + 1) % 3] = k & 1;
        off[(a + 2) % 3] = k >> 1;
        F.copies[8 * f + 4 * s + k] = cellnode[8 * cid + off[0] + 2 * off[1] + 4 * off[2]];
      }
    }
    F.ebar[f] = 0.5 * (E[F.cells[2 * f]] + E[F.cells[2 * f + 1]]);
    F.ups[f] = 2.0 * (kCf0 + ap * ap * ap / 12.0) / kMu;
  }
}

// ------------------------------------------------------------------ C1, Q1 (rows: copies)
// The fractured faces around grid node G in face-id order: normal d, plane
// G[d], in-plane cells (p, q) in {G[t1]-1, G[t1]} x {G[t2]-1, G[t2]}, q
// slower.  The copy is on the minus side of face f when the minus cell of f
// (bit d of its offset 0) is in its mask, on the plus side when the plus
// cell is; a copy on both sides (a fracture tip) has no jump and no entry.
template <int MODE, bool FILL>   // MODE 0: C1 (3x3), 1: Q1 (3x1)
__global__ void k_assemble_c1q1(Geo g, int nn, const int *copy_grid, const uint8_t *copy_mask, const int *fmap,
                                const int8_t *dir, int *cnt, const int *rp, int *ci, double *val) {
  const double w = g.h * g.h / 4.0;   // integral of a nodal basis over a face
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    const int gid = copy_grid[i];
    const int G[3] = {gid % g.N1, (gid / g.N1) % g.N1, gid / (g.N1 * g.N1)};
    const int mi = copy_mask[i];
    int k = FILL ? rp[i] : 0;
    for (int d = 0; d < 3; d++) {
      if (G[d] < 1 || G[d] > g.N - 1) continue;
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      for (int dq = -1; dq <= 0; dq++)
        for (int dp = -1; dp <= 0; dp++) {
          const int p = G[t1] + dp, q = G[t2] + dq;
          if (p < 0 || p >= g.N || q < 0 || q >= g.N) continue;
          const int f = fmap[g.fidx(d, G[d], p, q)];
          if (f < 0) continue;
          int bits[3];
          bits[d] = 0;
          bits[t1] = dp + 1;
          bits[t2] = dq + 1;
          const int em = bits[0] + 2 * bits[1] + 4 * bits[2];
          const int ep = em | (1 << d);
          const bool on_m = (mi >> em) & 1, on_p = (mi >> ep) & 1;
          if (on_m == on_p) continue;
          const double sg = on_p ? 1.0 : -1.0;
          double b[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
          bool nz = false;
          if (MODE == 0) {
            // C1 (copy, f)[c][r] = sg w R_f[r][c]: rows n, t1, t2 of the frame
            const int axis[3] = {d, t1, t2};
            for (int r = 0; r < 3; r++) {
              const int c = axis[r];
              if (!dir[3 * i + c]) {
                b[3 * c + r] = sg * w;
                nz = true;
              }
            }
          } else {
            if (!dir[3 * i + d]) {
              b[d] = -sg * w;
              nz = true;
            }
          }
          if (!nz) continue;   // every row of the block eliminated by a roller
          if (FILL) {
            ci[k] = f;
            const int bs = MODE == 0 ? 9 : 3;
            for (int t = 0; t < bs; t++) val[(int64_t)k * bs + t] = b[t];
          }
          k++;
        }
    }
    if (!FILL) cnt[i] = k;
  }
}

// ------------------------------------------------------------------ C2 (rows: faces)
// Eq. C2def: stick (mu, [[eta]]); slip (mu_N, [[eta_N]]) and
// -(1/k)(mu_T, dt_T*/dDg_T . [[eta_T]]) with t_T* = tau Dg_T / |Dg_T|,
// tau = c - t_N tan(theta), so dt_T*/dDg_T = (tau / |Dg_T|)(I - g g^T);
// open: none.  Columns: the face's copies in increasing id.
template <bool FILL>
__global__ void k_assemble_c2(int nf, double h, double kscale, double tan_th, const int *geom, FaceData F,
                              const int8_t *dir, int *cnt, const int *rp, int *ci, double *val) {
  const double w = h * h / 4.0;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int st = F.state[f];
    int k = FILL ? rp[f] : 0;
    if (st != 2) {
      const int a = geom[4 * f];
      const int axis[3] = {a, (a + 1) % 3, (a + 2) % 3};
      int cp[8];
      double sg[8];
      int n = 0;
      for (int c = 0; c < 4; c++) {
        const int m = F.copies[8 * f + c], p = F.copies[8 * f + 4 + c];
        if (m == p) continue;
        cp[n] = m; sg[n] = -1.0; n++;
        cp[n] = p; sg[n] = 1.0; n++;
      }
      for (int x = 1; x < n; x++)   // at most 8 columns: insertion sort by copy
        for (int y = x; y > 0 && cp[y - 1] > cp[y]; y--) {
          const int ti = cp[y]; cp[y] = cp[y - 1]; cp[y - 1] = ti;
          const double td = sg[y]; sg[y] = sg[y - 1]; sg[y - 1] = td;
        }
      const double kf = F.ebar[f] / (kscale * h);
      const double tau = -F.tn[f] * tan_th;
      const double g1 = F.g1[f], g2 = F.g2[f], sc = tau / F.dg[f];
      const double D[2][2] = {{sc * (1.0 - g1 * g1), -sc * g1 * g2}, {-sc * g1 * g2, sc * (1.0 - g2 * g2)}};
      for (int t = 0; t < n; t++) {
        const int c = cp[t];
        double b[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        b[axis[0]] = sg[t] * w;                      // normal row
        for (int r = 0; r < 2; r++)
          for (int x = 0; x < 2; x++) {
            const double v = st == 0 ? (r == x ? sg[t] * w : 0.0) : -sg[t] * (w / kf) * D[r][x];
            b[3 * (r + 1) + axis[x + 1]] += v;
          }
        bool nz = false;
        for (int r = 0; r < 3; r++)
          for (int x = 0; x < 3; x++) {
            if (dir[3 * c + x]) b[3 * r + x] = 0.0;
            nz |= b[3 * r + x] != 0.0;
          }
        if (!nz) continue;
        if (FILL) {
          ci[k] = c;
          for (int x = 0; x < 9; x++) val[(int64_t)k * 9 + x] = b[x];
        }
        k++;
      }
    }
    if (!FILL) cnt[f] = k;
  }
}

// ------------------------------------------------------------------ face neighbours
// The faces sharing each edge of face f.  An edge of f along axis `dir` at
// grid point E lies on four cell faces: for each normal d != dir, the faces
// at plane E[d] whose cells sit at E[o] - 1 or E[o] along the third axis o.
// nbr[12 f ..]: neighbour ids in increasing order (-1 padded), cop: 1 for a
// coplanar neighbour; ecnt[4 f + e]: fractured faces on edge e of f.
__global__ void k_face_neighbours(Geo g, int nf, const int *geom, const int *fmap, int *nbr, int8_t *cop,
                                  int8_t *ecnt) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int a = geom[4 * f], m = geom[4 * f + 1], p = geom[4 * f + 2], q = geom[4 * f + 3];
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    int ids[kMaxNbr];
    int8_t cp[kMaxNbr];
    int n = 0;
    for (int e = 0; e < 4; e++) {
      int E[3];
      E[a] = m;
      int dir;
      if (e < 2) { E[t1] = p; E[t2] = q + e; dir = t1; }
      else { E[t1] = p + (e - 2); E[t2] = q; dir = t2; }
      int on_edge = 0;
      for (int d = 0; d < 3; d++) {
        if (d == dir) continue;
        if (E[d] < 1 || E[d] > g.N - 1) continue;
        const int o = 3 - d - dir;
        for (int s = -1; s <= 0; s++) {
          int c[3];
          c[dir] = E[dir];
          c[o] = E[o] + s;
          if (c[o] < 0 || c[o] >= g.N) continue;
          const int L = fmap[g.fidx(d, E[d], c[(d + 1) % 3], c[(d + 2) % 3])];
          if (L < 0) continue;
          on_edge++;
          if (L == f) continue;
          ids[n] = L;
          cp[n] = d == a;
          n++;
        }
      }
      ecnt[4 * f + e] = (int8_t)on_edge;
    }
    for (int x = 1; x < n; x++)
      for (int y = x; y > 0 && ids[y - 1] > ids[y]; y--) {
        const int ti = ids[y]; ids[y] = ids[y - 1]; ids[y - 1] = ti;
        const int8_t tc = cp[y]; cp[y] = cp[y - 1]; cp[y - 1] = tc;
      }
    for (int x = 0; x < kMaxNbr; x++) {
      nbr[kMaxNbr * f + x] = x < n ? ids[x] : -1;
      cop[kMaxNbr * f + x] = x < n ? cp[x] : 0;
    }
  }
}

// Dirichlet pressure edges: for each fracture, its distinct corner faces;
// an edge of such a face on the fracture's outline that no other face
// touches carries p = 0.  dcnt[f] counts them (one thread per fracture).
__global__ void k_dirichlet_edges(Geo g, const Fracture *fr, int n_fr, const int *fmap, const int8_t *ecnt,
                                  int *dcnt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_fr) return;
  const Fracture F = fr[r];
  const int pq[4][2] = {{F.p0, F.q0}, {F.p1, F.q0}, {F.p0, F.q1}, {F.p1, F.q1}};
  int done[4];
  int nd = 0;
  for (int c = 0; c < 4; c++) {
    const int p = pq[c][0], q = pq[c][1];
    const int K = fmap[g.fidx(F.a, F.m, p, q)];
    bool dup = K < 0;
    for (int i = 0; i < nd; i++) dup |= done[i] == K;
    if (dup) continue;
    done[nd++] = K;
    for (int e = 0; e < 4; e++) {
      const bool outer = (e == 0 && q == F.q0) || (e == 1 && q == F.q1) || (e == 2 && p == F.p0) ||
                         (e == 3 && p == F.p1);
      if (outer && ecnt[4 * K + e] == 1) atomicAdd(&dcnt[K], 1);
    }
  }
}

// stabilisation tensor of the edge between coplanar faces K and L
struct Ups {
  double n, t;
};
__device__ inline Ups edge_ups(const FaceData &F, const double *E, int K, int L, double beta, double h) {
  const double Mfac = (1.0 - kNu) / ((1.0 + kNu) * (1.0 - 2.0 * kNu));   // M / E
  const double Gfac = 1.0 / (2.0 * (1.0 + kNu));                          // G / E
  const double Ebar4 = 0.25 * (E[F.cells[2 * K]] + E[F.cells[2 * K + 1]] + E[F.cells[2 * L]] + E[F.cells[2 * L + 1]]);
  return {beta * h * h * h / (Mfac * Ebar4), beta * h * h * h / (Gfac * Ebar4)};
}

// ------------------------------------------------------------------ T and H (rows: faces)
// T (Eq. Tdef): series TPFA over every pair sharing an edge, (1/dt) j_p on
// coplanar pairs (all states), one-sided transmissibility on Dirichlet
// edges.  H (Eq. Hdef): j_t on coplanar pairs of stick/slip faces (diagonal
// for each stick/slip face, off-diagonal when both are), -(1/k)(mu_T, mu_T)
// and (1/k)(mu_T, dt_T*/dt_N mu_N) on slip faces (dt_T*/dt_N = -tan(theta) g),
// -(1/k)(mu, mu) on open faces.
template <bool FILL>
__global__ void k_assemble_th(int nf, double h, double beta, double kscale, double tan_th, FaceData F,
                              const double *E, const int *nbr, const int8_t *cop, const int *dcnt, int *cntT,
                              int *cntH, const int *rpT, int *ciT, double *valT, const int *rpH, int *ciH,
                              double *valH) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int st = F.state[f];
    const bool act = st != 2;
    int kT = FILL ? rpT[f] : 0, kH = FILL ? rpH[f] : 0;
    double tdiag = 0.0, hd[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int diagT = -1, diagH = -1;
    bool placed = false;
    for (int x = 0; x <= kMaxNbr; x++) {
      const int L = x < kMaxNbr ? nbr[kMaxNbr * f + x] : -1;
      if (!placed && (L < 0 || L > f)) {   // the diagonal in its sorted place
        placed = true;
        diagT = kT++;
        diagH = kH++;
      }
      if (L < 0) break;
      const double uK = F.ups[f], uL = F.ups[L];
      const double uKL = uK * uL / (uK + uL);
      double t = -uKL;
      tdiag += uKL;
      if (cop[kMaxNbr * f + x]) {
        const Ups u = edge_ups(F, E, f, L, beta, h);
        t -= u.n / kDt;
        tdiag += u.n / kDt;
        if (act) {
          hd[0] += u.n; hd[4] += u.t; hd[8] += u.t;
          if (F.state[L] != 2) {
            if (FILL) {
              ciH[kH] = L;
              double *v = valH + (int64_t)kH * 9;
              for (int y = 0; y < 9; y++) v[y] = 0.0;
              v[0] = -u.n; v[4] = -u.t; v[8] = -u.t;
            }
            kH++;
          }
        }
      }
      if (FILL) {
        ciT[kT] = L;
        valT[kT] = t;
      }
      kT++;
    }
    if (FILL) {
      tdiag += dcnt[f] * F.ups[f];
      ciT[diagT] = f;
      valT[diagT] = tdiag;
      const double hk = h * h / (F.ebar[f] / (kscale * h));   // h^2 / k
      if (st == 1) {
        hd[4] += -hk; hd[8] += -hk;
        hd[3] += -hk * tan_th * F.g1[f];
        hd[6] += -hk * tan_th * F.g2[f];
      } else if (st == 2) {
        hd[0] += -hk; hd[4] += -hk; hd[8] += -hk;
      }
      ciH[diagH] = f;
      for (int y = 0; y < 9; y++) valH[(int64_t)diagH * 9 + y] = hd[y];
    } else {
      cntT[f] = kT;
      cntH[f] = kH;
    }
  }
}

// ------------------------------------------------------------------ Q2 (rows: faces)
// Eq. Q2def / Eq. Q2vsQ1: Q2 = -Psi(Q1^T) / dt + F_u.  F_u row K holds the
// derivative of the TPFA flux of face K through the open faces' apertures:
// for each neighbour L, (p_K - p_L) [Ups_L^2 / (Ups_K + Ups_L)^2 dUps_K/du +
// Ups_K^2 / (Ups_K + Ups_L)^2 dUps_L/du], and p_K dUps_K/du per Dirichlet
// edge; dUps_M/du = (2 / mu)(a_M^2 / 4) dg_M/du for open M, dg_M/du = +-n/4
// on M's plus / minus copies.  Every source face M contributes coef_M
// (+-1/4) n_M on its copies; the row's columns are the sources' copies in
// increasing id, each summed over the sources in a fixed order.
constexpr int kQ2Src = 1 + kMaxNbr;
template <bool FILL>
__global__ void k_assemble_q2(int nf, double h, FaceData F, const int *geom, const int *nbr, const int *dcnt,
                              const int8_t *dir, int *cnt, const int *rp, int *ci, double *val) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    int src[kQ2Src];
    double coef[kQ2Src];
    int ns = 0;
    const double uK = F.ups[f];
    const bool openK = F.state[f] == 2;
    double cK = 0.0;   // the row face's own coefficient of dUps_K/du
    for (int x = 0; x < kMaxNbr; x++) {
      const int L = nbr[kMaxNbr * f + x];
      if (L < 0) break;
      const double uL = F.ups[L], S = uK + uL;
      const double dp = F.pl[f] - F.pl[L];
      if (openK) cK += dp * (uL * uL / (S * S));
      if (F.state[L] == 2) {
        src[ns] = L;
        coef[ns] = dp * (uK * uK / (S * S)) * (2.0 / kMu) * (F.aper[L] * F.aper[L] / 4.0) * 0.25;
        ns++;
      }
    }
    if (openK) {
      cK += dcnt[f] * F.pl[f];
      src[ns] = f;
      coef[ns] = cK * (2.0 / kMu) * (F.aper[f] * F.aper[f] / 4.0) * 0.25;
      ns++;
    }
    // candidate columns: the non-tip copies of the sources, sorted, unique
    int cand[8 * kQ2Src];
    int nc = 0;
    for (int s = 0; s < ns; s++)
      for (int c = 0; c < 4; c++) {
        const int m = F.copies[8 * src[s] + c], p = F.copies[8 * src[s] + 4 + c];
        if (m == p) continue;
        cand[nc++] = m;
        cand[nc++] = p;
      }
    for (int x = 1; x < nc; x++)
      for (int y = x; y > 0 && cand[y - 1] > cand[y]; y--) {
        const int t = cand[y]; cand[y] = cand[y - 1]; cand[y - 1] = t;
      }
    int k = FILL ? rp[f] : 0;
    const double wdt = (h * h / 4.0) / kDt;
    for (int x = 0; x < nc; x++) {
      if (x > 0 && cand[x] == cand[x - 1]) continue;
      const int col = cand[x];
      double b[3] = {0.0, 0.0, 0.0};
      if (openK) {   // storage term (1/dt)(chi, [[eta_N]]) of the row face
        const int a = geom[4 * f];
        for (int c = 0; c < 4; c++) {
          const int m = F.copies[8 * f + c], p = F.copies[8 * f + 4 + c];
          if (m == p) continue;
          if (p == col) b[a] += wdt;
          if (m == col) b[a] -= wdt;
        }
      }
      for (int s = 0; s < ns; s++) {
        const int M = src[s], a = geom[4 * M];
        for (int c = 0; c < 4; c++) {
          const int m = F.copies[8 * M + c], p = F.copies[8 * M + 4 + c];
          if (m == p) continue;
          if (p == col) b[a] += coef[s];
          if (m == col) b[a] -= coef[s];
        }
      }
      bool nz = false;
      for (int c = 0; c < 3; c++) {
        if (dir[3 * col + c]) b[c] = 0.0;
        nz |= b[c] != 0.0;
      }
      if (!nz) continue;
      if (FILL) {
        ci[k] = col;
        for (int c = 0; c < 3; c++) val[(int64_t)k * 3 + c] = b[c];
      }
      k++;
    }
    if (!FILL) cnt[f] = k;
  }
}

__global__ void k_rhs(uint64_t seed, int64_t n, int64_t nu, const int8_t *dir, double *b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (i < nu && dir[i]) ? 0.0 : 2.0 * sm64_uniform(seed, S_RHS, (uint64_t)i) - 1.0;
}

// ------------------------------------------------------------------ host side
// 24x24 stiffness of the unit trilinear hexahedron, E = 1 (isotropic Hooke,
// 2x2x2 Gauss points, exact for the cube); corner a at (a & 1, a >> 1 & 1,
// a >> 2 & 1), dof 3 a + component.
std::vector<double> hex8_unit_stiffness(double nu) {
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), G = 1.0 / (2.0 * (1.0 + nu));
  std::vector<double> K(576, 0.0);
  const double gp[2] = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
  for (int gz = 0; gz < 2; gz++)
    for (int gy = 0; gy < 2; gy++)
      for (int gx = 0; gx < 2; gx++) {
        const double X[3] = {gp[gx], gp[gy], gp[gz]};
        double dN[8][3];   // gradients of the shape functions
        for (int a = 0; a < 8; a++) {
          const int o[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
          double f[3], df[3];
          for (int d = 0; d < 3; d++) {
            f[d] = o[d] ? X[d] : 1.0 - X[d];
            df[d] = o[d] ? 1.0 : -1.0;
          }
          dN[a][0] = df[0] * f[1] * f[2];
          dN[a][1] = f[0] * df[1] * f[2];
          dN[a][2] = f[0] * f[1] * df[2];
        }
        const double wgt = 0.125;   // (1/2)^3 per point on the unit cube
        // K_ab[i][j] = lam dN_a[i] dN_b[j] + G (dN_a[j] dN_b[i] + delta_ij dN_a . dN_b)
        for (int a = 0; a < 8; a++)
          for (int b = 0; b < 8; b++) {
            const double dd = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2];
            for (int i = 0; i < 3; i++)
              for (int j = 0; j < 3; j++)
                K[(3 * a + i) * 24 + 3 * b + j] +=
                    wgt * (lam * dN[a][i] * dN[b][j] + G * dN[a][j] * dN[b][i] + (i == j ? G * dd : 0.0));
          }
      }
  return K;
}

std::vector<Fracture> fractures(const fc_gen_config &c, uint64_t seed) {
  const int N = c.N;
  std::vector<Fracture> fr;
  if (c.layout == FC_GEN_PLANE_X) {
    fr.push_back({0, N / 2, 0, 0, N - 1, N - 1});
  } else if (c.layout == FC_GEN_PLANES_XYZ) {
    for (int a = 0; a < 3; a++) fr.push_back({a, N / 2, 0, 0, N - 1, N - 1});
  } else if (c.layout == FC_GEN_RECTS) {
    for (int r = 0; r < c.n_rect; r++) {
      const uint64_t i0 = 8 * (uint64_t)r;
      const int a = (int)std::floor(3.0 * sm64_uniform(seed, S_RECT, i0 + 0));
      const int m = 1 + (int)std::floor((N - 1) * sm64_uniform(seed, S_RECT, i0 + 1));
      const int e1 = std::max(1, (int)std::lround(N * (0.2 + 0.6 * sm64_uniform(seed, S_RECT, i0 + 2))));
      const int e2 = std::max(1, (int)std::lround(N * (0.2 + 0.6 * sm64_uniform(seed, S_RECT, i0 + 3))));
      const int p0 = (int)std::floor((N - e1 + 1) * sm64_uniform(seed, S_RECT, i0 + 4));
      const int q0 = (int)std::floor((N - e2 + 1) * sm64_uniform(seed, S_RECT, i0 + 5));
      fr.push_back({a, m, p0, q0, p0 + e1 - 1, q0 + e2 - 1});
    }
  } else if (c.layout == FC_GEN_NETWORK) {
    for (int a = 0; a < 3; a++)
      for (int m = c.spacing; m <= N - 1; m += c.spacing) fr.push_back({a, m, 0, 0, N - 1, N - 1});
  }
  return fr;
}

thread_local std::string g_gen_err;

}  // namespace

// The instance and everything it owns on the device.
struct GenInstance {
  fc_instance pub;
  Bsr<double> A, C1, Q1, C2, H, Q2, T;
  DBuf<double> b, aper, pl, ebar;
  DBuf<int8_t> state, dir;
  DBuf<int> geom, copies, node_grid;
};

namespace {

void set_block(fc_bsr &d, const Bsr<double> &m) {
  d.n_brows = m.nbr; d.n_bcols = m.nbc; d.br = m.br; d.bc = m.bc; d.nnzb = m.nnzb;
  d.d_row_ptr = m.rp.p; d.d_col_idx = m.ci.p; d.d_val = m.val.p;
}

// count pass -> row pointers -> storage (the fill pass is the caller's)
void alloc_rows(Bsr<double> &M, int nbr, int nbc, int br, int bc, const DBuf<int> &cnt, cudaStream_t s) {
  M.shape(nbr, nbc, br, bc);
  M.rp.alloc((size_t)nbr + 1);
  M.nnzb = nbr > 0 ? exclusive_scan(cnt.p, M.rp.p, nbr, s) : 0;
  if (nbr == 0) FS_CUDA(cudaMemsetAsync(M.rp.p, 0, sizeof(int), s));
  M.ci.alloc((size_t)std::max<int64_t>(M.nnzb, 1));
  M.val.alloc((size_t)std::max<int64_t>(M.nnzb, 1) * br * bc);
}

GenInstance *generate(const fc_gen_config &c, uint64_t seed, cudaStream_t s) {
  FS_REQUIRE(c.N >= 2 && c.N <= 1024, FC_BAD_ARG, "fc_generate: N must lie in [2, 1024]");
  FS_REQUIRE(c.layout >= FC_GEN_PLANE_X && c.layout <= FC_GEN_NETWORK, FC_BAD_ARG, "fc_generate: unknown layout");
  FS_REQUIRE(c.layout != FC_GEN_NETWORK || c.spacing >= 1, FC_BAD_ARG, "fc_generate: spacing must be >= 1");
  FS_REQUIRE(c.layout != FC_GEN_RECTS || (c.n_rect >= 0 && c.n_rect <= 4096), FC_BAD_ARG,
             "fc_generate: n_rect must lie in [0, 4096]");
  FS_REQUIRE(c.p_stick >= 0 && c.p_slip >= 0 && c.p_stick + c.p_slip <= 1.0, FC_BAD_ARG,
             "fc_generate: state probabilities must be >= 0 with p_stick + p_slip <= 1");
  FS_REQUIRE(std::isfinite(c.sigma_E) && std::isfinite(c.aperture_sigma) && std::isfinite(c.pl_scale), FC_BAD_ARG,
             "fc_generate: non-finite parameter");
  const int N = c.N, N1 = N + 1;
  const double h = 1.0 / N;
  const double beta = c.beta > 0 ? c.beta : 0.25;
  const double kscale = c.k_scale > 0 ? c.k_scale : 8.0;
  const double tan_th = std::tan(30.0 * M_PI / 180.0);
  Geo g{N, N1, h};
  auto out = std::make_unique<GenInstance>();

  // fractures and faces
  const std::vector<Fracture> frh = fractures(c, seed);
  const int n_fr = (int)frh.size();
  FS_REQUIRE(!c.d_aperture || c.n_aperture >= 0, FC_BAD_ARG, "fc_generate: negative n_aperture");
  DBuf<Fracture> fr(std::max(n_fr, 1));
  if (n_fr) FS_CUDA(cudaMemcpyAsync(fr.p, frh.data(), sizeof(Fracture) * n_fr, cudaMemcpyHostToDevice, s));
  const int64_t nslot = (int64_t)3 * N1 * N * N;
  FS_REQUIRE(nslot < INT32_MAX, FC_BAD_ARG, "fc_generate: grid too large");
  DBuf<int> flag(nslot), pre(nslot + 1), fmap(nslot);
  k_face_flags<<<blocks_for(nslot, 256), 256, 0, s>>>(g, fr.p, n_fr, flag.p);
  FS_LAUNCHED();
  const int nf = (int)exclusive_scan(flag.p, pre.p, (int)nslot, s);
  FS_REQUIRE(!c.d_aperture || c.n_aperture == nf, FC_BAD_ARG,
             "fc_generate: n_aperture = " + std::to_string(c.n_aperture) + " but the layout has " +
                 std::to_string(nf) + " fracture faces");
  out->geom.alloc((size_t)4 * std::max(nf, 1));
  k_face_ids<<<blocks_for(nslot, 256), 256, 0, s>>>(g, flag.p, pre.p, fmap.p, out->geom.p);
  FS_LAUNCHED();
  flag.release();
  pre.release();

  // node split
  const int64_t ngrid = (int64_t)N1 * N1 * N1, ncell = (int64_t)N * N * N;
  DBuf<int> ncnt(ngrid), first(ngrid + 1);
  k_node_count<<<blocks_for(ngrid, 256), 256, 0, s>>>(g, fmap.p, ncnt.p);
  FS_LAUNCHED();
  const int nn = (int)exclusive_scan(ncnt.p, first.p, (int)ngrid, s);
  ncnt.release();
  out->node_grid.alloc(nn);
  DBuf<uint8_t> mask(nn);
  DBuf<int> cellnode(8 * ncell);
  k_node_split<<<blocks_for(ngrid, 256), 256, 0, s>>>(g, fmap.p, first.p, out->node_grid.p, mask.p, cellnode.p);
  FS_LAUNCHED();
  DBuf<double> E(ncell);
  k_material<<<blocks_for(ncell, 256), 256, 0, s>>>(g, seed, c.sigma_E, E.p);
  FS_LAUNCHED();
  out->dir.alloc((size_t)3 * nn);
  k_dirichlet<<<blocks_for(nn, 256), 256, 0, s>>>(g, out->node_grid.p, nn, out->dir.p);
  FS_LAUNCHED();

  // A
  const std::vector<double> kh = hex8_unit_stiffness(kNu);
  DBuf<double> Khat(576);
  FS_CUDA(cudaMemcpyAsync(Khat.p, kh.data(), sizeof(double) * 576, cudaMemcpyHostToDevice, s));
  {
    DBuf<int> cnt(nn);
    k_assemble_A<false><<<blocks_for(nn, 128), 128, 0, s>>>(g, nn, out->node_grid.p, mask.p, first.p, E.p, Khat.p,
                                                            out->dir.p, cnt.p, nullptr, nullptr, nullptr);
    FS_LAUNCHED();
    alloc_rows(out->A, nn, nn, 3, 3, cnt, s);
    k_assemble_A<true><<<blocks_for(nn, 128), 128, 0, s>>>(g, nn, out->node_grid.p, mask.p, first.p, E.p, Khat.p,
                                                           out->dir.p, nullptr, out->A.rp.p, out->A.ci.p,
                                                           out->A.val.p);
    FS_LAUNCHED();
  }
  // C1, Q1
  {
    DBuf<int> cnt(std::max(nn, 1));
    k_assemble_c1q1<0, false><<<blocks_for(nn, 256), 256, 0, s>>>(g, nn, out->node_grid.p, mask.p, fmap.p,
                                                                  out->dir.p, cnt.p, nullptr, nullptr, nullptr);
    FS_LAUNCHED();
    alloc_rows(out->C1, nn, nf, 3, 3, cnt, s);
    k_assemble_c1q1<0, true><<<blocks_for(nn, 256), 256, 0, s>>>(g, nn, out->node_grid.p, mask.p, fmap.p,
                                                                 out->dir.p, nullptr, out->C1.rp.p, out->C1.ci.p,
                                                                 out->C1.val.p);
    FS_LAUNCHED();
    k_assemble_c1q1<1, false><<<blocks_for(nn, 256), 256, 0, s>>>(g, nn, out->node_grid.p, mask.p, fmap.p,
                                                                  out->dir.p, cnt.p, nullptr, nullptr, nullptr);
    FS_LAUNCHED();
    alloc_rows(out->Q1, nn, nf, 3, 1, cnt, s);
    k_assemble_c1q1<1, true><<<blocks_for(nn, 256), 256, 0, s>>>(g, nn, out->node_grid.p, mask.p, fmap.p,
                                                                 out->dir.p, nullptr, out->Q1.rp.p, out->Q1.ci.p,
                                                                 out->Q1.val.p);
    FS_LAUNCHED();
  }

  // per-face data
  const int nfa = std::max(nf, 1);
  out->state.alloc(nfa);
  out->aper.alloc(nfa);
  out->pl.alloc(nfa);
  out->ebar.alloc(nfa);
  out->copies.alloc((size_t)8 * nfa);
  DBuf<double> ups(nfa), tn(nfa), g1(nfa), g2(nfa), dg(nfa);
  DBuf<int64_t> fcells((size_t)2 * nfa);
  FaceData F{out->state.p, out->aper.p, out->pl.p, out->ebar.p, ups.p, tn.p, g1.p, g2.p, dg.p, out->copies.p,
             fcells.p};
  if (nf)
    k_face_data<<<blocks_for(nf, 256), 256, 0, s>>>(g, nf, out->geom.p, cellnode.p, E.p, seed, c.p_stick, c.p_slip,
                                                    c.aperture_sigma, c.d_aperture, c.pl_scale, F);
  if (nf) FS_LAUNCHED();
  // C2
  {
    DBuf<int> cnt(nfa);
    if (nf) {
      k_assemble_c2<false><<<blocks_for(nf, 256), 256, 0, s>>>(nf, h, kscale, tan_th, out->geom.p, F, out->dir.p,
                                                               cnt.p, nullptr, nullptr, nullptr);
      FS_LAUNCHED();
    }
    alloc_rows(out->C2, nf, nn, 3, 3, cnt, s);
    if (nf) {
      k_assemble_c2<true><<<blocks_for(nf, 256), 256, 0, s>>>(nf, h, kscale, tan_th, out->geom.p, F, out->dir.p,
                                                              nullptr, out->C2.rp.p, out->C2.ci.p, out->C2.val.p);
      FS_LAUNCHED();
    }
  }
  // neighbours, H, T, Q2
  {
    DBuf<int> nbr((size_t)kMaxNbr * nfa), dcnt(nfa), cT(nfa), cH(nfa), cQ(nfa);
    DBuf<int8_t> cop((size_t)kMaxNbr * nfa), ecnt((size_t)4 * nfa);
    FS_CUDA(cudaMemsetAsync(dcnt.p, 0, sizeof(int) * nfa, s));
    if (nf) {
      k_face_neighbours<<<blocks_for(nf, 256), 256, 0, s>>>(g, nf, out->geom.p, fmap.p, nbr.p, cop.p, ecnt.p);
      FS_LAUNCHED();
      if (n_fr) {
        k_dirichlet_edges<<<(n_fr + 63) / 64, 64, 0, s>>>(g, fr.p, n_fr, fmap.p, ecnt.p, dcnt.p);
        FS_LAUNCHED();
      }
      k_assemble_th<false><<<blocks_for(nf, 128), 128, 0, s>>>(nf, h, beta, kscale, tan_th, F, E.p, nbr.p, cop.p,
                                                               dcnt.p, cT.p, cH.p, nullptr, nullptr, nullptr,
                                                               nullptr, nullptr, nullptr);
      FS_LAUNCHED();
      k_assemble_q2<false><<<blocks_for(nf, 128), 128, 0, s>>>(nf, h, F, out->geom.p, nbr.p, dcnt.p, out->dir.p,
                                                               cQ.p, nullptr, nullptr, nullptr);
      FS_LAUNCHED();
    }
    alloc_rows(out->T, nf, nf, 1, 1, cT, s);
    alloc_rows(out->H, nf, nf, 3, 3, cH, s);
    alloc_rows(out->Q2, nf, nn, 1, 3, cQ, s);
    if (nf) {
      k_assemble_th<true><<<blocks_for(nf, 128), 128, 0, s>>>(nf, h, beta, kscale, tan_th, F, E.p, nbr.p, cop.p,
                                                              dcnt.p, nullptr, nullptr, out->T.rp.p, out->T.ci.p,
                                                              out->T.val.p, out->H.rp.p, out->H.ci.p, out->H.val.p);
      FS_LAUNCHED();
      k_assemble_q2<true><<<blocks_for(nf, 128), 128, 0, s>>>(nf, h, F, out->geom.p, nbr.p, dcnt.p, out->dir.p,
                                                              nullptr, out->Q2.rp.p, out->Q2.ci.p, out->Q2.val.p);
      FS_LAUNCHED();
    }
  }
  // right-hand side
  const int64_t n = 3 * (int64_t)nn + 4 * (int64_t)nf;
  out->b.alloc(n);
  k_rhs<<<blocks_for(n, 256), 256, 0, s>>>(seed, n, 3 * (int64_t)nn, out->dir.p, out->b.p);
  FS_LAUNCHED();
  FS_CUDA(cudaStreamSynchronize(s));   // the temporaries are freed on return

  fc_instance &P = out->pub;
  std::memset(&P, 0, sizeof(P));
  set_block(P.J.A, out->A); set_block(P.J.C1, out->C1); set_block(P.J.Q1, out->Q1);
  set_block(P.J.C2, out->C2); set_block(P.J.H, out->H); set_block(P.J.Q2, out->Q2);
  set_block(P.J.T, out->T);
  P.J.n_node = nn;
  P.J.n_face = nf;
  P.n_node = nn;
  P.n_face = nf;
  P.n = n;
  P.grid_n = N;
  P.d_b = out->b.p;
  P.d_state = out->state.p;
  P.d_dirichlet = out->dir.p;
  P.d_aperture = out->aper.p;
  P.d_pl = out->pl.p;
  P.d_ebar = out->ebar.p;
  P.d_face_geom = out->geom.p;
  P.d_face_copies = out->copies.p;
  P.d_node_grid = out->node_grid.p;
  P.h = h;
  P.dt = kDt;
  P.nu = kNu;
  P.owner = out.get();
  return out.release();
}

}  // namespace
}  // namespace fs

extern "C" {

void fc_default_gen_config(fc_gen_config *c, int layout, int N) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->N = N;
  c->layout = layout;
  c->p_stick = 0.6;
  c->p_slip = 0.3;
  c->sigma_E = 1.0;
  c->aperture_sigma = 0.5;
  c->pl_scale = 1.0;
  if (layout == FC_GEN_PLANE_X) {
    c->p_stick = 1.0;
    c->p_slip = 0.0;
    c->sigma_E = 0.5;
    c->aperture_sigma = 0.0;
  } else if (layout == FC_GEN_RECTS) {
    c->n_rect = 10;
  } else if (layout == FC_GEN_NETWORK) {
    c->spacing = 8;
    c->p_stick = 0.5;
    c->p_slip = 0.4;
  }
}

int fc_generate(const fc_gen_config *cfg, uint64_t seed, void *cuda_stream, fc_instance **out) {
  if (!cfg || !out) return FC_BAD_ARG;
  *out = nullptr;
  fs::g_gen_err.clear();
  try {
    fs::GenInstance *g = fs::generate(*cfg, seed, static_cast<cudaStream_t>(cuda_stream));
    *out = &g->pub;
    return FC_OK;
  } catch (const fs::Error &e) {
    fs::g_gen_err = e.what();
    (void)cudaGetLastError();
    return e.code;
  } catch (const std::bad_alloc &) {
    fs::g_gen_err = "host allocation failed";
    return FC_OOM;
  } catch (const std::exception &e) {
    fs::g_gen_err = e.what();
    return FC_INTERNAL;
  }
}

const char *fc_generate_error(void) { return fs::g_gen_err.c_str(); }

void fc_instance_free(fc_instance *inst) {
  if (!inst) return;
  delete static_cast<fs::GenInstance *>(inst->owner);
}

}  // extern "C"
