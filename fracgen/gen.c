/*
 * fracgen: seeded synthetic generator of the linearised 3x3 block Jacobian of
 * frictional contact mechanics with flow in a fracture network
 * (Franceschini, Gazzola, Ferronato, arXiv 2112.12397, Sec. 2, Eq. JacSys and
 * Eq. block_def).
 *
 * This module produces INPUTS only.  It holds none of the solver's arithmetic
 * (no Schur complement, no preconditioner, no Krylov method); both the CPU
 * oracle and the CUDA library consume what it writes.
 *
 * Unknowns (Sec. 2.1): u = 3 displacement components per node copy (global
 * frame), t = 3 traction components per fracture face (local frame n, t1, t2),
 * p = 1 pressure per fracture face.  The vector order is [u; t; p].
 *
 * Blocks (Eq. block_def):
 *   A  (n_node x n_node, 3x3)  trilinear hex stiffness, 2x2x2 Gauss
 *   C1 (n_node x n_face, 3x3)  (jump(eta), mu)_Gamma
 *   Q1 (n_node x n_face, 3x1)  -(jump(eta_N), chi)_Gamma
 *   C2 (n_face x n_node, 3x3)  stick: C1^T; slip: normal row + friction
 *                              derivative rows; open: 0
 *   H  (n_face x n_face, 3x3)  -(1/k) slip/open terms + j_t stabilisation
 *   Q2 (n_face x n_node, 1x3)  (1/dt)(chi, jump(eta_N))_open + dF/du (TPFA)
 *   T  (n_face x n_face, 1x1)  TPFA transmissibility + (1/dt) j_p
 * The Jacobian is [A C1 Q1; C2 -H 0; Q2 0 T].
 *
 * Where the paper leaves a quantity unspecified (stabilisation tensor, k,
 * boundary conditions, material field, slip data, flow at intersections) the
 * reading used here is stated at the point where it is applied.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* counter-based random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA'14) */
/* ------------------------------------------------------------------------ */
#define FG_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t fg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* r(seed, stream, i): output i+1 of a SplitMix64 sequence whose state starts
 * at key = mix64(seed*gamma + stream). */
uint64_t fg_rand_u64(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t key = fg_mix64(seed * FG_GAMMA + stream);
  return fg_mix64(key + (i + 1) * FG_GAMMA);
}

/* U in [0, 1) with 53 random bits */
double fg_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(fg_rand_u64(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* standard normal by Box-Muller from draws 2i and 2i+1 */
double fg_normal(uint64_t seed, uint64_t stream, uint64_t i) {
  double u1 = 1.0 - fg_uniform(seed, stream, 2 * i);      /* (0, 1] */
  double u2 = fg_uniform(seed, stream, 2 * i + 1);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

enum {
  ST_E = 1, ST_STATE = 2, ST_TN = 3, ST_PHI = 4, ST_DG = 5, ST_APER = 6,
  ST_PL = 7, ST_RHS = 8, ST_RECT = 9
};

/* ------------------------------------------------------------------------ */
/* public structures                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t N;            /* cells per axis of the unit cube */
  int32_t layout;       /* 0: x-plane at N/2; 1: x,y,z planes at N/2;
                           2: n_rect seeded rectangles; 3: planes every
                           `spacing` cells on all three axes */
  int32_t n_rect;
  int32_t spacing;
  double p_stick, p_slip;   /* state probabilities; open = rest */
  double sigma_E;           /* lognormal spread of Young's modulus */
  double aperture_sigma;    /* 0: aperture = 1e-3 m everywhere */
  uint64_t seed;
  const double *aperture_in;  /* optional n_face apertures (m); NULL = draw */
  double beta;              /* stabilisation scale; <= 0 selects the default */
  double k_scale;           /* k = Ebar_f / (k_scale h); <= 0 selects default */
  double pl_scale;          /* multiplies the drawn current pressures p^l */
} fg_config;

typedef struct {
  int32_t n_brows, n_bcols, br, bc;
  int64_t nnzb;
  int32_t *row_ptr, *col_idx;
  double *val;
} fg_bsr;

typedef struct {
  int32_t N, n_node, n_face, n_rect_eff;
  double h, dt, mu, E0, nu, C_f0, beta, tan_theta;
  fg_bsr A, C1, Q1, C2, H, Q2, T;
  double *b;             /* 3 n_node + 4 n_face */
  int8_t *state;         /* n_face: 0 stick, 1 slip, 2 open */
  int8_t *dirichlet;     /* 3 n_node */
  int32_t *node_grid;    /* n_node: grid node id (i + (N+1)(j + (N+1)k)) */
  int32_t *face_geom;    /* 4 n_face: axis, m, p, q */
  int32_t *face_copies;  /* 8 n_face: minus copies (4 corners) then plus */
  double *aperture, *pl, *E_cell, *Ebar_face, *ups_face;
  int32_t *rects;        /* 5 per fracture: axis, m, p0, q0, p1, (q1 in
                            rects_q1) */
  int32_t *rects_q1;
  /* derivatives of the Jacobian with respect to the apertures: entry e says
   * d K[row, col] / d a_face = val, where for block 0 (T) row and col are
   * faces (comp = 0) and for block 1 (Q2) row is a face and (col, comp) a
   * displacement dof (copy, component).  Sorted by (face, block, row, col,
   * comp), duplicates summed. */
  int64_t n_dk;
  int32_t *dk_face, *dk_row, *dk_col;
  int8_t *dk_block, *dk_comp;
  double *dk_val;
} fg_problem;

/* ------------------------------------------------------------------------ */
/* growable COO of small dense blocks and its conversion to BSR              */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n, cap;
  int bsz;
  int32_t *r, *c;
  double *v;
} coo_t;

static void coo_init(coo_t *q, int bsz) {
  q->n = 0; q->cap = 1024; q->bsz = bsz;
  q->r = (int32_t *)malloc(sizeof(int32_t) * q->cap);
  q->c = (int32_t *)malloc(sizeof(int32_t) * q->cap);
  q->v = (double *)malloc(sizeof(double) * q->cap * bsz);
}
static double *coo_push(coo_t *q, int32_t r, int32_t c) {
  if (q->n == q->cap) {
    q->cap *= 2;
    q->r = (int32_t *)realloc(q->r, sizeof(int32_t) * q->cap);
    q->c = (int32_t *)realloc(q->c, sizeof(int32_t) * q->cap);
    q->v = (double *)realloc(q->v, sizeof(double) * q->cap * q->bsz);
  }
  q->r[q->n] = r; q->c[q->n] = c;
  double *v = q->v + q->n * q->bsz;
  memset(v, 0, sizeof(double) * q->bsz);
  q->n++;
  return v;
}
static void coo_free(coo_t *q) { free(q->r); free(q->c); free(q->v); }

/* Rows sorted by column, duplicates summed.  drop_zero: remove blocks whose
 * entries are all exactly zero. */
static void coo_to_bsr(coo_t *q, int32_t nr, int32_t nc, int br, int bc,
                       int drop_zero, fg_bsr *out) {
  int bsz = br * bc;
  int32_t *cnt = (int32_t *)calloc((size_t)nr + 1, sizeof(int32_t));
  for (int64_t e = 0; e < q->n; e++) cnt[q->r[e] + 1]++;
  for (int32_t i = 0; i < nr; i++) cnt[i + 1] += cnt[i];
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (q->n > 0 ? q->n : 1));
  int32_t *fill = (int32_t *)calloc((size_t)nr, sizeof(int32_t));
  for (int64_t e = 0; e < q->n; e++) {
    int32_t r = q->r[e];
    perm[cnt[r] + fill[r]++] = e;
  }
  /* per-row insertion sort by column (rows are short) */
  for (int32_t i = 0; i < nr; i++) {
    int64_t s = cnt[i], t = cnt[i + 1];
    for (int64_t a = s + 1; a < t; a++) {
      int64_t key = perm[a];
      int64_t b = a - 1;
      while (b >= s && q->c[perm[b]] > q->c[key]) { perm[b + 1] = perm[b]; b--; }
      perm[b + 1] = key;
    }
  }
  out->n_brows = nr; out->n_bcols = nc; out->br = br; out->bc = bc;
  out->row_ptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nr + 1));
  int64_t cap = q->n > 0 ? q->n : 1;
  int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * cap);
  double *vv = (double *)malloc(sizeof(double) * cap * bsz);
  int64_t nnz = 0;
  out->row_ptr[0] = 0;
  for (int32_t i = 0; i < nr; i++) {
    int64_t s = cnt[i], t = cnt[i + 1];
    int64_t a = s;
    while (a < t) {
      int32_t col = q->c[perm[a]];
      double acc[16];
      memset(acc, 0, sizeof(acc));
      while (a < t && q->c[perm[a]] == col) {
        const double *v = q->v + perm[a] * bsz;
        for (int k = 0; k < bsz; k++) acc[k] += v[k];
        a++;
      }
      int nonzero = 0;
      for (int k = 0; k < bsz; k++) nonzero |= (acc[k] != 0.0);
      if (drop_zero && !nonzero) continue;
      ci[nnz] = col;
      memcpy(vv + nnz * bsz, acc, sizeof(double) * bsz);
      nnz++;
    }
    out->row_ptr[i + 1] = (int32_t)nnz;
  }
  out->nnzb = nnz;
  out->col_idx = ci;
  out->val = vv;
  free(cnt); free(perm); free(fill);
}

static void bsr_free(fg_bsr *m) {
  free(m->row_ptr); free(m->col_idx); free(m->val);
  m->row_ptr = NULL; m->col_idx = NULL; m->val = NULL;
}

/* ------------------------------------------------------------------------ */
/* derivative entries d K / d a_face                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n, cap;
  int32_t *face, *row, *col;
  int8_t *block, *comp;
  double *val;
} dk_t;

static void dk_init(dk_t *d) {
  d->n = 0; d->cap = 1024;
  d->face = (int32_t *)malloc(sizeof(int32_t) * d->cap);
  d->row = (int32_t *)malloc(sizeof(int32_t) * d->cap);
  d->col = (int32_t *)malloc(sizeof(int32_t) * d->cap);
  d->block = (int8_t *)malloc(d->cap);
  d->comp = (int8_t *)malloc(d->cap);
  d->val = (double *)malloc(sizeof(double) * d->cap);
}
static void dk_push(dk_t *d, int32_t f, int block, int32_t row, int32_t col, int comp, double v) {
  if (v == 0.0) return;
  if (d->n == d->cap) {
    d->cap *= 2;
    d->face = (int32_t *)realloc(d->face, sizeof(int32_t) * d->cap);
    d->row = (int32_t *)realloc(d->row, sizeof(int32_t) * d->cap);
    d->col = (int32_t *)realloc(d->col, sizeof(int32_t) * d->cap);
    d->block = (int8_t *)realloc(d->block, d->cap);
    d->comp = (int8_t *)realloc(d->comp, d->cap);
    d->val = (double *)realloc(d->val, sizeof(double) * d->cap);
  }
  d->face[d->n] = f; d->block[d->n] = (int8_t)block; d->row[d->n] = row;
  d->col[d->n] = col; d->comp[d->n] = (int8_t)comp; d->val[d->n] = v;
  d->n++;
}
static const dk_t *g_dk_sort;
static int cmp_dk(const void *a, const void *b) {
  int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
  const dk_t *d = g_dk_sort;
#define CMPF(x) if (d->x[i] != d->x[j]) return d->x[i] < d->x[j] ? -1 : 1;
  CMPF(face) CMPF(block) CMPF(row) CMPF(col) CMPF(comp)
#undef CMPF
  return (i > j) - (i < j);
}

/* ------------------------------------------------------------------------ */
/* element stiffness of the unit trilinear hexahedron, E = 1, h = 1          */
/* ------------------------------------------------------------------------ */
/* local node a = dx + 2 dy + 4 dz, reference coordinate 2d - 1 */
void fg_hex8_stiffness(double nu, double *Ke /* 24 x 24 row-major */) {
  double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double G = 1.0 / (2.0 * (1.0 + nu));
  double D[6][6];
  memset(D, 0, sizeof(D));
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) D[i][j] = lam;
    D[i][i] = lam + 2.0 * G;
    D[3 + i][3 + i] = G;
  }
  memset(Ke, 0, sizeof(double) * 576);
  const double g = 1.0 / sqrt(3.0);
  for (int gp = 0; gp < 8; gp++) {
    double xi = (gp & 1) ? g : -g, eta = (gp & 2) ? g : -g, ze = (gp & 4) ? g : -g;
    double dN[8][3];
    for (int a = 0; a < 8; a++) {
      double xa = (a & 1) ? 1.0 : -1.0, ya = (a & 2) ? 1.0 : -1.0, za = (a & 4) ? 1.0 : -1.0;
      /* derivative w.r.t. physical coords on [0,1]^3: d/dx = 2 d/dxi */
      dN[a][0] = 2.0 * 0.125 * xa * (1 + ya * eta) * (1 + za * ze);
      dN[a][1] = 2.0 * 0.125 * ya * (1 + xa * xi) * (1 + za * ze);
      dN[a][2] = 2.0 * 0.125 * za * (1 + xa * xi) * (1 + ya * eta);
    }
    double B[6][24];
    memset(B, 0, sizeof(B));
    for (int a = 0; a < 8; a++) {
      double dx = dN[a][0], dy = dN[a][1], dz = dN[a][2];
      B[0][3 * a + 0] = dx;
      B[1][3 * a + 1] = dy;
      B[2][3 * a + 2] = dz;
      B[3][3 * a + 0] = dy; B[3][3 * a + 1] = dx;   /* gamma_xy */
      B[4][3 * a + 1] = dz; B[4][3 * a + 2] = dy;   /* gamma_yz */
      B[5][3 * a + 0] = dz; B[5][3 * a + 2] = dx;   /* gamma_zx */
    }
    double DB[6][24];
    for (int i = 0; i < 6; i++)
      for (int j = 0; j < 24; j++) {
        double s = 0;
        for (int k = 0; k < 6; k++) s += D[i][k] * B[k][j];
        DB[i][j] = s;
      }
    const double detJ = 0.125;   /* (1/2)^3, Gauss weights are 1 */
    for (int i = 0; i < 24; i++)
      for (int j = 0; j < 24; j++) {
        double s = 0;
        for (int k = 0; k < 6; k++) s += B[k][i] * DB[k][j];
        Ke[i * 24 + j] += s * detJ;
      }
  }
}

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */
static int uf_find(int *p, int x) { while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; } return x; }

typedef struct { int64_t key; int32_t face; int32_t pad; } edge_rec;
static int cmp_edge(const void *a, const void *b) {
  const edge_rec *x = (const edge_rec *)a, *y = (const edge_rec *)b;
  if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
  return (x->face > y->face) - (x->face < y->face);
}

/* ------------------------------------------------------------------------ */
/* main entry                                                                */
/* ------------------------------------------------------------------------ */
int fg_generate(const fg_config *cfg, fg_problem *P) {
  memset(P, 0, sizeof(*P));
  const int N = cfg->N;
  if (N < 2) return 1;
  const int N1 = N + 1;
  const uint64_t seed = cfg->seed;
  /* constants: MPa, m, s (the paper's test cases use MPa and s) */
  const double h = 1.0 / N;
  const double E0 = 1.0e4;              /* 10 GPa */
  const double nu = 0.25;
  const double mu = 1.0e-9;             /* 1e-3 Pa s in MPa s */
  const double dt = 0.5;                /* time step of the paper's tests */
  const double C_f0 = 9.87e-15;         /* conductivity of closed faces, m^3 */
  /* Reading (the paper defers the stabilisation tensor and k to its
   * reference [fr2020alg]): Upsilon^(eps) = beta h^3 diag(1/M, 1/G, 1/G) in
   * the local frame with M, G from the mean E of the four cells beside the
   * edge, and k = Ebar_f / (k_scale h).  With beta = 1/4 and k_scale = 8 the
   * tangential diagonal of a slip block is at most (20 beta - k_scale) h^3/Ebar
   * = -3 h^3/Ebar, so every slip block of H~ is non-singular. */
  const double beta = cfg->beta > 0 ? cfg->beta : 0.25;
  const double kfac = cfg->k_scale > 0 ? cfg->k_scale : 8.0;
  const double tan_theta = tan(30.0 * M_PI / 180.0);
  P->N = N; P->h = h; P->dt = dt; P->mu = mu; P->E0 = E0; P->nu = nu;
  P->C_f0 = C_f0; P->beta = beta; P->tan_theta = tan_theta;

  /* ---------------- fractures: list of rectangles (axis, m, p0..p1, q0..q1) */
  int n_fr = 0;
  int32_t *fr = NULL;   /* 6 per fracture */
  if (cfg->layout == 0) {
    n_fr = 1; fr = (int32_t *)malloc(6 * sizeof(int32_t));
    int32_t r0[6] = {0, N / 2, 0, 0, N - 1, N - 1};
    memcpy(fr, r0, sizeof(r0));
  } else if (cfg->layout == 1) {
    n_fr = 3; fr = (int32_t *)malloc(18 * sizeof(int32_t));
    for (int a = 0; a < 3; a++) {
      int32_t r0[6] = {a, N / 2, 0, 0, N - 1, N - 1};
      memcpy(fr + 6 * a, r0, sizeof(r0));
    }
  } else if (cfg->layout == 2) {
    n_fr = cfg->n_rect; fr = (int32_t *)malloc(6 * sizeof(int32_t) * (n_fr > 0 ? n_fr : 1));
    for (int r = 0; r < n_fr; r++) {
      uint64_t i0 = 8 * (uint64_t)r;
      int a = (int)floor(3.0 * fg_uniform(seed, ST_RECT, i0 + 0));
      int m = 1 + (int)floor((N - 1) * fg_uniform(seed, ST_RECT, i0 + 1));
      int e1 = (int)lround(N * (0.2 + 0.6 * fg_uniform(seed, ST_RECT, i0 + 2)));
      int e2 = (int)lround(N * (0.2 + 0.6 * fg_uniform(seed, ST_RECT, i0 + 3)));
      if (e1 < 1) e1 = 1;
      if (e2 < 1) e2 = 1;
      int p0 = (int)floor((N - e1 + 1) * fg_uniform(seed, ST_RECT, i0 + 4));
      int q0 = (int)floor((N - e2 + 1) * fg_uniform(seed, ST_RECT, i0 + 5));
      int32_t r0[6] = {a, m, p0, q0, p0 + e1 - 1, q0 + e2 - 1};
      memcpy(fr + 6 * r, r0, sizeof(r0));
    }
  } else if (cfg->layout == 3) {
    int s = cfg->spacing;
    if (s < 1) return 1;
    int per = 0;
    for (int m = s; m <= N - 1; m += s) per++;
    n_fr = 3 * per; fr = (int32_t *)malloc(6 * sizeof(int32_t) * (n_fr > 0 ? n_fr : 1));
    int k = 0;
    for (int a = 0; a < 3; a++)
      for (int m = s; m <= N - 1; m += s) {
        int32_t r0[6] = {a, m, 0, 0, N - 1, N - 1};
        memcpy(fr + 6 * k, r0, sizeof(r0)); k++;
      }
  } else {
    return 1;
  }

  /* face map: fmap[((a*N1 + m)*N + q)*N + p] = face id or -1; a face is
   * owned by the lowest fracture index that covers it */
  const int64_t fmap_n = (int64_t)3 * N1 * N * N;
  int32_t *fmap = (int32_t *)malloc(sizeof(int32_t) * fmap_n);
  int32_t *fowner = (int32_t *)malloc(sizeof(int32_t) * fmap_n);
  for (int64_t i = 0; i < fmap_n; i++) { fmap[i] = -1; fowner[i] = -1; }
  for (int r = 0; r < n_fr; r++) {
    int a = fr[6 * r], m = fr[6 * r + 1];
    for (int q = fr[6 * r + 3]; q <= fr[6 * r + 5]; q++)
      for (int p = fr[6 * r + 2]; p <= fr[6 * r + 4]; p++) {
        int64_t k = (((int64_t)a * N1 + m) * N + q) * N + p;
        if (fowner[k] < 0) fowner[k] = r;
      }
  }
#define FIDX(a, m, p, q) ((((int64_t)(a) * N1 + (m)) * N + (q)) * N + (p))
  /* lexicographic (a, m, q, p) numbering */
  int32_t nf = 0;
  for (int64_t k = 0; k < fmap_n; k++)
    if (fowner[k] >= 0) fmap[k] = nf++;
  P->n_face = nf;
  P->face_geom = (int32_t *)malloc(sizeof(int32_t) * 4 * (nf > 0 ? nf : 1));
  for (int a = 0; a < 3; a++)
    for (int m = 0; m < N1; m++)
      for (int q = 0; q < N; q++)
        for (int p = 0; p < N; p++) {
          int32_t f = fmap[FIDX(a, m, p, q)];
          if (f < 0) continue;
          P->face_geom[4 * f + 0] = a; P->face_geom[4 * f + 1] = m;
          P->face_geom[4 * f + 2] = p; P->face_geom[4 * f + 3] = q;
        }
  P->n_rect_eff = n_fr;
  P->rects = (int32_t *)malloc(sizeof(int32_t) * 5 * (n_fr > 0 ? n_fr : 1));
  P->rects_q1 = (int32_t *)malloc(sizeof(int32_t) * (n_fr > 0 ? n_fr : 1));
  for (int r = 0; r < n_fr; r++) {
    for (int k = 0; k < 5; k++) P->rects[5 * r + k] = fr[6 * r + k];
    P->rects_q1[r] = fr[6 * r + 5];
  }

  /* ---------------- node split (DFM, nodes duplicated across fractures) */
  const int64_t ncell = (int64_t)N * N * N;
  const int64_t ngrid = (int64_t)N1 * N1 * N1;
  int32_t *cellnode = (int32_t *)malloc(sizeof(int32_t) * 8 * ncell);
  int64_t copy_cap = ngrid + 16;
  int32_t *copy_grid = (int32_t *)malloc(sizeof(int32_t) * copy_cap);
  int32_t ncopy = 0;
  for (int K = 0; K < N1; K++)
    for (int J = 0; J < N1; J++)
      for (int I = 0; I < N1; I++) {
        int gid = I + N1 * (J + N1 * K);
        int G[3] = {I, J, K};
        int valid[8]; int64_t cid[8]; int par[8];
        for (int e = 0; e < 8; e++) {
          int c[3] = {I - 1 + (e & 1), J - 1 + ((e >> 1) & 1), K - 1 + ((e >> 2) & 1)};
          valid[e] = c[0] >= 0 && c[0] < N && c[1] >= 0 && c[1] < N && c[2] >= 0 && c[2] < N;
          cid[e] = valid[e] ? c[0] + (int64_t)N * (c[1] + (int64_t)N * c[2]) : -1;
          par[e] = e;
        }
        for (int e = 0; e < 8; e++) {
          if (!valid[e]) continue;
          for (int d = 0; d < 3; d++) {
            if (e & (1 << d)) continue;
            int e2 = e | (1 << d);
            if (!valid[e2]) continue;
            /* shared face: normal d at plane G[d]; in-plane coords are the
             * common cell coords along (d+1)%3 and (d+2)%3 */
            int c[3] = {I - 1 + (e & 1), J - 1 + ((e >> 1) & 1), K - 1 + ((e >> 2) & 1)};
            int p = c[(d + 1) % 3], q = c[(d + 2) % 3];
            if (fmap[FIDX(d, G[d], p, q)] >= 0) continue;   /* fractured */
            int r1 = uf_find(par, e), r2 = uf_find(par, e2);
            if (r1 != r2) par[r1] = r2;
          }
        }
        /* components ordered by smallest incident cell id */
        int64_t cmin[8]; int root_of[8];
        for (int e = 0; e < 8; e++) cmin[e] = INT64_MAX;
        for (int e = 0; e < 8; e++) {
          if (!valid[e]) continue;
          int r = uf_find(par, e);
          root_of[e] = r;
          if (cid[e] < cmin[r]) cmin[r] = cid[e];
        }
        int roots[8], nroot = 0;
        for (int e = 0; e < 8; e++) if (valid[e] && uf_find(par, e) == e) roots[nroot++] = e;
        for (int a = 1; a < nroot; a++) {
          int key = roots[a], b = a - 1;
          while (b >= 0 && cmin[roots[b]] > cmin[key]) { roots[b + 1] = roots[b]; b--; }
          roots[b + 1] = key;
        }
        int copy_of_root[8];
        for (int a = 0; a < nroot; a++) {
          if (ncopy >= copy_cap) {
            copy_cap *= 2;
            copy_grid = (int32_t *)realloc(copy_grid, sizeof(int32_t) * copy_cap);
          }
          copy_grid[ncopy] = gid;
          copy_of_root[roots[a]] = ncopy++;
        }
        for (int e = 0; e < 8; e++) {
          if (!valid[e]) continue;
          int loc = (1 - (e & 1)) + 2 * (1 - ((e >> 1) & 1)) + 4 * (1 - ((e >> 2) & 1));
          cellnode[8 * cid[e] + loc] = copy_of_root[root_of[e]];
        }
      }
  const int32_t nn = ncopy;
  P->n_node = nn;
  P->node_grid = copy_grid;

  /* ---------------- material field: median-E0 lognormal per cell */
  P->E_cell = (double *)malloc(sizeof(double) * ncell);
  for (int64_t c = 0; c < ncell; c++)
    P->E_cell[c] = E0 * exp(cfg->sigma_E * fg_normal(seed, ST_E, (uint64_t)c));

  /* ---------------- boundary conditions: rollers on the six outer faces */
  P->dirichlet = (int8_t *)calloc((size_t)3 * nn, 1);
  for (int32_t i = 0; i < nn; i++) {
    int g = copy_grid[i];
    int G[3] = {g % N1, (g / N1) % N1, g / (N1 * N1)};
    for (int d = 0; d < 3; d++)
      if (G[d] == 0 || G[d] == N) P->dirichlet[3 * i + d] = 1;
  }
  const int8_t *dir = P->dirichlet;

  /* ---------------- A: BSR over node copies */
  {
    /* copy -> cells */
    int32_t *cc_cnt = (int32_t *)calloc((size_t)nn + 1, sizeof(int32_t));
    for (int64_t s = 0; s < 8 * ncell; s++) cc_cnt[cellnode[s] + 1]++;
    for (int32_t i = 0; i < nn; i++) cc_cnt[i + 1] += cc_cnt[i];
    int32_t *cc = (int32_t *)malloc(sizeof(int32_t) * 8 * ncell);
    int32_t *cfill = (int32_t *)calloc((size_t)nn, sizeof(int32_t));
    for (int64_t s = 0; s < 8 * ncell; s++) {
      int32_t i = cellnode[s];
      cc[cc_cnt[i] + cfill[i]++] = (int32_t)(s / 8);
    }
    free(cfill);
    int32_t *rp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nn + 1));
    rp[0] = 0;
    /* pass 1: row lengths */
    for (int pass = 0; pass < 2; pass++) {
      int32_t *ci = NULL;
      if (pass == 1) {
        ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)rp[nn]);
        P->A.col_idx = ci;
      }
      for (int32_t i = 0; i < nn; i++) {
        int32_t cand[64]; int nc = 0;
        for (int32_t t = cc_cnt[i]; t < cc_cnt[i + 1]; t++) {
          int32_t c = cc[t];
          for (int a = 0; a < 8; a++) cand[nc++] = cellnode[8 * (int64_t)c + a];
        }
        for (int a = 1; a < nc; a++) {
          int32_t key = cand[a]; int b = a - 1;
          while (b >= 0 && cand[b] > key) { cand[b + 1] = cand[b]; b--; }
          cand[b + 1] = key;
        }
        int nu_ = 0;
        for (int a = 0; a < nc; a++)
          if (a == 0 || cand[a] != cand[a - 1]) cand[nu_++] = cand[a];
        if (pass == 0) rp[i + 1] = rp[i] + nu_;
        else memcpy(ci + rp[i], cand, sizeof(int32_t) * nu_);
      }
    }
    free(cc); free(cc_cnt);
    P->A.n_brows = nn; P->A.n_bcols = nn; P->A.br = 3; P->A.bc = 3;
    P->A.row_ptr = rp; P->A.nnzb = rp[nn];
    P->A.val = (double *)calloc((size_t)rp[nn] * 9, sizeof(double));
    double Khat[576];
    fg_hex8_stiffness(nu, Khat);
    for (int64_t c = 0; c < ncell; c++) {
      double s = P->E_cell[c] * h;
      for (int a = 0; a < 8; a++) {
        int32_t row = cellnode[8 * c + a];
        const int32_t *cols = P->A.col_idx + rp[row];
        int len = rp[row + 1] - rp[row];
        for (int b = 0; b < 8; b++) {
          int32_t col = cellnode[8 * c + b];
          int lo = 0, hi = len - 1;
          while (lo < hi) { int mid = (lo + hi) / 2; if (cols[mid] < col) lo = mid + 1; else hi = mid; }
          double *blk = P->A.val + ((int64_t)rp[row] + lo) * 9;
          for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) blk[3 * i + j] += s * Khat[(3 * a + i) * 24 + 3 * b + j];
        }
      }
    }
    /* symmetric elimination of constrained dofs (keep the diagonal) */
    for (int32_t r = 0; r < nn; r++)
      for (int32_t k = rp[r]; k < rp[r + 1]; k++) {
        int32_t c = P->A.col_idx[k];
        double *blk = P->A.val + (int64_t)k * 9;
        for (int i = 0; i < 3; i++)
          for (int j = 0; j < 3; j++)
            if ((dir[3 * r + i] || dir[3 * c + j]) && !(r == c && i == j)) blk[3 * i + j] = 0.0;
      }
  }

  /* ---------------- per-face data */
  P->state = (int8_t *)malloc((size_t)(nf > 0 ? nf : 1));
  P->aperture = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  P->pl = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  P->Ebar_face = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  P->ups_face = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  P->face_copies = (int32_t *)malloc(sizeof(int32_t) * 8 * (nf > 0 ? nf : 1));
  double *tN = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  double *ghat = (double *)malloc(sizeof(double) * 2 * (nf > 0 ? nf : 1));
  double *dgn = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  int64_t *fcell = (int64_t *)malloc(sizeof(int64_t) * 2 * (nf > 0 ? nf : 1));
  for (int32_t f = 0; f < nf; f++) {
    int a = P->face_geom[4 * f], m = P->face_geom[4 * f + 1];
    int p = P->face_geom[4 * f + 2], q = P->face_geom[4 * f + 3];
    double U = fg_uniform(seed, ST_STATE, f);
    P->state[f] = U < cfg->p_stick ? 0 : (U < cfg->p_stick + cfg->p_slip ? 1 : 2);
    if (cfg->aperture_in) P->aperture[f] = cfg->aperture_in[f];
    else P->aperture[f] = 1e-3 * exp(cfg->aperture_sigma * fg_normal(seed, ST_APER, f));
    P->pl[f] = cfg->pl_scale * fg_uniform(seed, ST_PL, f);
    tN[f] = -(5.0 + 10.0 * fg_uniform(seed, ST_TN, f));
    double phi = 2.0 * M_PI * fg_uniform(seed, ST_PHI, f);
    ghat[2 * f] = cos(phi); ghat[2 * f + 1] = sin(phi);
    dgn[f] = 1e-4 * exp(0.5 * fg_normal(seed, ST_DG, f));
    for (int side = 0; side < 2; side++) {
      int c[3];
      c[a] = m - 1 + side; c[(a + 1) % 3] = p; c[(a + 2) % 3] = q;
      fcell[2 * f + side] = c[0] + (int64_t)N * (c[1] + (int64_t)N * c[2]);
      /* corner k = dp + 2 dq; node offset along a is 1 for the minus cell */
      for (int k = 0; k < 4; k++) {
        int dp = k & 1, dq = k >> 1;
        int off[3];
        off[a] = 1 - side; off[(a + 1) % 3] = dp; off[(a + 2) % 3] = dq;
        int loc = off[0] + 2 * off[1] + 4 * off[2];
        P->face_copies[8 * f + 4 * side + k] = cellnode[8 * fcell[2 * f + side] + loc];
      }
    }
    P->Ebar_face[f] = 0.5 * (P->E_cell[fcell[2 * f]] + P->E_cell[fcell[2 * f + 1]]);
    double Cf = C_f0 + P->aperture[f] * P->aperture[f] * P->aperture[f] / 12.0;
    /* one-sided transmissibility: (C_f / mu) |edge| / d_K, d_K = h / 2 */
    P->ups_face[f] = 2.0 * Cf / mu;
  }

  /* ---------------- C1, Q1 (rows: copies) and C2 (rows: faces) */
  {
    coo_t c1, q1, c2;
    coo_init(&c1, 9); coo_init(&q1, 3); coo_init(&c2, 9);
    const double w = h * h / 4.0;   /* integral of a nodal basis over a face */
    for (int32_t f = 0; f < nf; f++) {
      int a = P->face_geom[4 * f];
      double R[3][3];   /* rows n, t1, t2 in global coordinates */
      memset(R, 0, sizeof(R));
      R[0][a] = 1.0; R[1][(a + 1) % 3] = 1.0; R[2][(a + 2) % 3] = 1.0;
      double k_f = P->Ebar_face[f] / (kfac * h);
      double tau = -tN[f] * tan_theta;            /* c = 0 */
      double g1 = ghat[2 * f], g2 = ghat[2 * f + 1];
      double Dm[2][2] = {{tau / dgn[f] * (1 - g1 * g1), -tau / dgn[f] * g1 * g2},
                         {-tau / dgn[f] * g1 * g2, tau / dgn[f] * (1 - g2 * g2)}};
      for (int k = 0; k < 4; k++) {
        int32_t cm = P->face_copies[8 * f + k], cp = P->face_copies[8 * f + 4 + k];
        if (cm == cp) continue;   /* tip: continuous basis, zero jump */
        for (int side = 0; side < 2; side++) {
          int32_t cpy = side ? cp : cm;
          double sg = side ? 1.0 : -1.0;
          /* C1 block (copy, f)[c][d] = sg w R[d][c] */
          double *v = coo_push(&c1, cpy, f);
          for (int c = 0; c < 3; c++)
            for (int d = 0; d < 3; d++) v[3 * c + d] = sg * w * R[d][c];
          /* Q1 block (copy, f)[c] = -sg w n[c] */
          v = coo_push(&q1, cpy, f);
          v[a] = -sg * w;
          if (P->state[f] == 0) {           /* stick: C1^T */
            v = coo_push(&c2, f, cpy);
            for (int d = 0; d < 3; d++)
              for (int c = 0; c < 3; c++) v[3 * d + c] = sg * w * R[d][c];
          } else if (P->state[f] == 1) {    /* slip */
            v = coo_push(&c2, f, cpy);
            for (int c = 0; c < 3; c++) v[c] = sg * w * R[0][c];
            for (int d = 0; d < 2; d++)
              for (int c = 0; c < 3; c++)
                v[3 * (d + 1) + c] = -sg * (w / k_f) * (Dm[d][0] * R[1][c] + Dm[d][1] * R[2][c]);
          }
        }
      }
    }
    /* zero constrained rows of C1, Q1 and constrained columns of C2 */
    for (int64_t e = 0; e < c1.n; e++)
      for (int c = 0; c < 3; c++)
        if (dir[3 * c1.r[e] + c]) for (int d = 0; d < 3; d++) c1.v[9 * e + 3 * c + d] = 0.0;
    for (int64_t e = 0; e < q1.n; e++)
      for (int c = 0; c < 3; c++)
        if (dir[3 * q1.r[e] + c]) q1.v[3 * e + c] = 0.0;
    for (int64_t e = 0; e < c2.n; e++)
      for (int c = 0; c < 3; c++)
        if (dir[3 * c2.c[e] + c]) for (int d = 0; d < 3; d++) c2.v[9 * e + 3 * d + c] = 0.0;
    coo_to_bsr(&c1, nn, nf, 3, 3, 1, &P->C1);
    coo_to_bsr(&q1, nn, nf, 3, 1, 1, &P->Q1);
    coo_to_bsr(&c2, nf, nn, 3, 3, 1, &P->C2);
    coo_free(&c1); coo_free(&q1); coo_free(&c2);
  }

  /* ---------------- face edges: which faces share each grid edge */
  int64_t nrec = 4 * (int64_t)nf;
  edge_rec *er = (edge_rec *)malloc(sizeof(edge_rec) * (nrec > 0 ? nrec : 1));
  for (int32_t f = 0; f < nf; f++) {
    int a = P->face_geom[4 * f], m = P->face_geom[4 * f + 1];
    int p = P->face_geom[4 * f + 2], q = P->face_geom[4 * f + 3];
    int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    for (int e = 0; e < 4; e++) {
      int g[3]; int dirn;
      g[a] = m;
      if (e < 2) { g[t1] = p; g[t2] = q + e; dirn = t1; }       /* along t1 */
      else { g[t1] = p + (e - 2); g[t2] = q; dirn = t2; }       /* along t2 */
      int64_t gid = g[0] + (int64_t)N1 * (g[1] + (int64_t)N1 * g[2]);
      er[4 * f + e].key = gid * 3 + dirn;
      er[4 * f + e].face = f;
    }
  }
  qsort(er, (size_t)nrec, sizeof(edge_rec), cmp_edge);

  /* ---------------- H (3x3 per face pair), T (1x1), Q2 (1x3) */
  dk_t dk;
  dk_init(&dk);
  {
    coo_t hq, tq, q2;
    coo_init(&hq, 9); coo_init(&tq, 1); coo_init(&q2, 3);
    const double Mfac = (1.0 - nu) / ((1.0 + nu) * (1.0 - 2.0 * nu));   /* M / E */
    const double Gfac = 1.0 / (2.0 * (1.0 + nu));                       /* G / E */
    /* diagonal slip/open terms and structural diagonal */
    for (int32_t f = 0; f < nf; f++) {
      double *v = coo_push(&hq, f, f);
      double hk = h * h / (P->Ebar_face[f] / (kfac * h));   /* h^2 / k */
      if (P->state[f] == 1) {
        v[4] += -hk; v[8] += -hk;
        v[3] += -hk * tan_theta * ghat[2 * f];
        v[6] += -hk * tan_theta * ghat[2 * f + 1];
      } else if (P->state[f] == 2) {
        v[0] += -hk; v[4] += -hk; v[8] += -hk;
      }
      double *t = coo_push(&tq, f, f);
      (void)t;
    }
    /* d(Upsilon_M)/du for open M: (2/mu)(a^2/4) * dg/du, dg/du = +-n/4 */
    #define ADD_DUPS(row, M, coef)                                            \
      do {                                                                    \
        if (P->state[M] == 2) {                                               \
          double cM = (coef) * (2.0 / mu) * (P->aperture[M] * P->aperture[M] / 4.0) * 0.25; \
          int aM = P->face_geom[4 * (M)];                                     \
          for (int kk = 0; kk < 4; kk++) {                                    \
            int32_t cmn = P->face_copies[8 * (M) + kk], cpl = P->face_copies[8 * (M) + 4 + kk]; \
            if (cmn == cpl) continue;                                         \
            double *vv = coo_push(&q2, row, cpl); vv[aM] += cM;               \
            vv = coo_push(&q2, row, cmn); vv[aM] -= cM;                       \
          }                                                                   \
        }                                                                     \
      } while (0)
    /* derivative helper: d/d a_fc of coef * dg_M/du added to Q2 row `row` */
    #define ADD_DG(fc, row, M, coef)                                          \
      do {                                                                    \
        if (P->state[M] == 2) {                                               \
          int aM_ = P->face_geom[4 * (M)];                                    \
          for (int kk_ = 0; kk_ < 4; kk_++) {                                 \
            int32_t cm_ = P->face_copies[8 * (M) + kk_], cp_ = P->face_copies[8 * (M) + 4 + kk_]; \
            if (cm_ == cp_) continue;                                         \
            dk_push(&dk, fc, 1, row, cp_, aM_, 0.25 * (coef));                \
            dk_push(&dk, fc, 1, row, cm_, aM_, -0.25 * (coef));               \
          }                                                                   \
        }                                                                     \
      } while (0)
    int64_t s = 0;
    while (s < nrec) {
      int64_t t = s;
      while (t < nrec && er[t].key == er[s].key) t++;
      int ng = (int)(t - s);
      for (int64_t i = s; i < t; i++)
        for (int64_t j = i + 1; j < t; j++) {
          int32_t K = er[i].face, L = er[j].face;
          double uK = P->ups_face[K], uL = P->ups_face[L];
          double uKL = uK * uL / (uK + uL);
          double *v;
          v = coo_push(&tq, K, K); v[0] += uKL;
          v = coo_push(&tq, L, L); v[0] += uKL;
          v = coo_push(&tq, K, L); v[0] -= uKL;
          v = coo_push(&tq, L, K); v[0] -= uKL;
          /* F_u: rows K and L of d/du [Ups_KL (p_K - p_L)] */
          double dK = uL * uL / ((uK + uL) * (uK + uL));
          double dL = uK * uK / ((uK + uL) * (uK + uL));
          double dp = P->pl[K] - P->pl[L];
          ADD_DUPS(K, K, dp * dK); ADD_DUPS(K, L, dp * dL);
          ADD_DUPS(L, K, -dp * dK); ADD_DUPS(L, L, -dp * dL);
          {
            /* d/da of the transmissibility entries and of the flux
             * derivative rows; Ups_M = 2 (C_f0 + a_M^3 / 12) / mu, so
             * dUps_M/da_M = cM = (2 / mu)(a_M^2 / 4) and dcM/da_M = a_M / mu */
            const double aK = P->aperture[K], aL = P->aperture[L];
            const double cK = (2.0 / mu) * (aK * aK / 4.0), cL = (2.0 / mu) * (aL * aL / 4.0);
            const double S = uK + uL, S3 = S * S * S;
            const double tK = dK * cK, tL = dL * cL;
            dk_push(&dk, K, 0, K, K, 0, tK); dk_push(&dk, K, 0, L, L, 0, tK);
            dk_push(&dk, K, 0, K, L, 0, -tK); dk_push(&dk, K, 0, L, K, 0, -tK);
            dk_push(&dk, L, 0, K, K, 0, tL); dk_push(&dk, L, 0, L, L, 0, tL);
            dk_push(&dk, L, 0, K, L, 0, -tL); dk_push(&dk, L, 0, L, K, 0, -tL);
            /* V = dK cK G_K + dL cL G_L; rows K (x dp) and L (x -dp) */
            const double vKK = cK * cK * (-2.0 * uL * uL / S3) + dK * aK / mu;   /* dV/daK on G_K */
            const double vKL = cK * cL * (2.0 * uK * uL / S3);                   /* dV/daK on G_L */
            const double vLK = cK * cL * (2.0 * uK * uL / S3);                   /* dV/daL on G_K */
            const double vLL = cL * cL * (-2.0 * uK * uK / S3) + dL * aL / mu;   /* dV/daL on G_L */
            ADD_DG(K, K, K, dp * vKK); ADD_DG(K, K, L, dp * vKL);
            ADD_DG(K, L, K, -dp * vKK); ADD_DG(K, L, L, -dp * vKL);
            ADD_DG(L, K, K, dp * vLK); ADD_DG(L, K, L, dp * vLL);
            ADD_DG(L, L, K, -dp * vLK); ADD_DG(L, L, L, -dp * vLL);
          }
          int coplanar = P->face_geom[4 * K] == P->face_geom[4 * L] &&
                         P->face_geom[4 * K + 1] == P->face_geom[4 * L + 1];
          if (coplanar) {
            double Ebar4 = 0.25 * (P->E_cell[fcell[2 * K]] + P->E_cell[fcell[2 * K + 1]] +
                                   P->E_cell[fcell[2 * L]] + P->E_cell[fcell[2 * L + 1]]);
            double uN = beta * h * h * h / (Mfac * Ebar4);
            double uT = beta * h * h * h / (Gfac * Ebar4);
            /* j_p: normal projection of j_t, scaled by 1/dt, all states */
            v = coo_push(&tq, K, K); v[0] += uN / dt;
            v = coo_push(&tq, L, L); v[0] += uN / dt;
            v = coo_push(&tq, K, L); v[0] -= uN / dt;
            v = coo_push(&tq, L, K); v[0] -= uN / dt;
            /* j_t over stick and slip faces */
            int aK = P->state[K] != 2, aL = P->state[L] != 2;
            if (aK) { v = coo_push(&hq, K, K); v[0] += uN; v[4] += uT; v[8] += uT; }
            if (aL) { v = coo_push(&hq, L, L); v[0] += uN; v[4] += uT; v[8] += uT; }
            if (aK && aL) {
              v = coo_push(&hq, K, L); v[0] -= uN; v[4] -= uT; v[8] -= uT;
              v = coo_push(&hq, L, K); v[0] -= uN; v[4] -= uT; v[8] -= uT;
            }
          }
        }
      (void)ng;
      s = t;
    }
    /* Dirichlet p = 0 on the outer edges of the four corner faces of every
     * fracture: edges on the fracture's boundary touched by no other face */
    for (int r = 0; r < n_fr; r++) {
      int a = fr[6 * r], m = fr[6 * r + 1];
      int p0 = fr[6 * r + 2], q0 = fr[6 * r + 3], p1 = fr[6 * r + 4], q1 = fr[6 * r + 5];
      int cps[4][2] = {{p0, q0}, {p1, q0}, {p0, q1}, {p1, q1}};
      int32_t done[4]; int nd = 0;
      for (int c = 0; c < 4; c++) {
        int32_t K = fmap[FIDX(a, m, cps[c][0], cps[c][1])];
        int dup = 0;
        for (int i = 0; i < nd; i++) dup |= (done[i] == K);
        if (dup || K < 0) continue;
        done[nd++] = K;
        int p = cps[c][0], q = cps[c][1];
        int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
        for (int e = 0; e < 4; e++) {
          int g[3]; int dirn; int outer;
          g[a] = m;
          if (e < 2) { g[t1] = p; g[t2] = q + e; dirn = t1; outer = (e == 0 && q == q0) || (e == 1 && q == q1); }
          else { g[t1] = p + (e - 2); g[t2] = q; dirn = t2; outer = (e == 2 && p == p0) || (e == 3 && p == p1); }
          if (!outer) continue;
          int64_t key = (g[0] + (int64_t)N1 * (g[1] + (int64_t)N1 * g[2])) * 3 + dirn;
          /* count faces on this edge */
          int64_t lo = 0, hi = nrec;
          while (lo < hi) { int64_t mid = (lo + hi) / 2; if (er[mid].key < key) lo = mid + 1; else hi = mid; }
          int cnt = 0;
          for (int64_t i = lo; i < nrec && er[i].key == key; i++) cnt++;
          if (cnt != 1) continue;
          double *v = coo_push(&tq, K, K); v[0] += P->ups_face[K];
          ADD_DUPS(K, K, P->pl[K]);
          {
            const double aK = P->aperture[K];
            dk_push(&dk, K, 0, K, K, 0, (2.0 / mu) * (aK * aK / 4.0));
            ADD_DG(K, K, K, P->pl[K] * aK / mu);
          }
        }
      }
    }
    /* open-face storage term of Q2: (1/dt)(chi, jump(eta_N)) = -Q1^T / dt */
    for (int32_t f = 0; f < nf; f++) {
      if (P->state[f] != 2) continue;
      int a = P->face_geom[4 * f];
      for (int k = 0; k < 4; k++) {
        int32_t cm = P->face_copies[8 * f + k], cp = P->face_copies[8 * f + 4 + k];
        if (cm == cp) continue;
        double *v = coo_push(&q2, f, cp); v[a] += (h * h / 4.0) / dt;
        v = coo_push(&q2, f, cm); v[a] -= (h * h / 4.0) / dt;
      }
    }
    #undef ADD_DUPS
    #undef ADD_DG
    for (int64_t e = 0; e < q2.n; e++)
      for (int c = 0; c < 3; c++)
        if (dir[3 * q2.c[e] + c]) q2.v[3 * e + c] = 0.0;
    coo_to_bsr(&hq, nf, nf, 3, 3, 0, &P->H);
    coo_to_bsr(&tq, nf, nf, 1, 1, 0, &P->T);
    coo_to_bsr(&q2, nf, nn, 1, 3, 1, &P->Q2);
    coo_free(&hq); coo_free(&tq); coo_free(&q2);
  }

  /* ---------------- derivative entries: drop constrained Q2 columns, sort,
   * merge duplicates */
  {
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (dk.n > 0 ? dk.n : 1));
    for (int64_t e = 0; e < dk.n; e++) perm[e] = e;
    g_dk_sort = &dk;
    qsort(perm, (size_t)dk.n, sizeof(int64_t), cmp_dk);
    int64_t m = 0;
    P->dk_face = (int32_t *)malloc(sizeof(int32_t) * (dk.n > 0 ? dk.n : 1));
    P->dk_row = (int32_t *)malloc(sizeof(int32_t) * (dk.n > 0 ? dk.n : 1));
    P->dk_col = (int32_t *)malloc(sizeof(int32_t) * (dk.n > 0 ? dk.n : 1));
    P->dk_block = (int8_t *)malloc(dk.n > 0 ? dk.n : 1);
    P->dk_comp = (int8_t *)malloc(dk.n > 0 ? dk.n : 1);
    P->dk_val = (double *)malloc(sizeof(double) * (dk.n > 0 ? dk.n : 1));
    for (int64_t t = 0; t < dk.n; t++) {
      int64_t e = perm[t];
      if (dk.block[e] == 1 && dir[3 * dk.col[e] + dk.comp[e]]) continue;
      if (m > 0 && P->dk_face[m - 1] == dk.face[e] && P->dk_block[m - 1] == dk.block[e] &&
          P->dk_row[m - 1] == dk.row[e] && P->dk_col[m - 1] == dk.col[e] && P->dk_comp[m - 1] == dk.comp[e]) {
        P->dk_val[m - 1] += dk.val[e];
        continue;
      }
      P->dk_face[m] = dk.face[e]; P->dk_block[m] = dk.block[e]; P->dk_row[m] = dk.row[e];
      P->dk_col[m] = dk.col[e]; P->dk_comp[m] = dk.comp[e]; P->dk_val[m] = dk.val[e];
      m++;
    }
    P->n_dk = m;
    free(perm);
    free(dk.face); free(dk.row); free(dk.col); free(dk.block); free(dk.comp); free(dk.val);
  }

  /* ---------------- right-hand side */
  {
    int64_t n = 3 * (int64_t)nn + 4 * (int64_t)nf;
    P->b = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; i++) P->b[i] = 2.0 * fg_uniform(seed, ST_RHS, (uint64_t)i) - 1.0;
    for (int64_t i = 0; i < 3 * (int64_t)nn; i++) if (dir[i]) P->b[i] = 0.0;
  }

  free(er); free(tN); free(ghat); free(dgn); free(fcell);
  free(fmap); free(fowner); free(cellnode); free(fr);
#undef FIDX
  return 0;
}

void fg_free(fg_problem *P) {
  bsr_free(&P->A); bsr_free(&P->C1); bsr_free(&P->Q1); bsr_free(&P->C2);
  bsr_free(&P->H); bsr_free(&P->Q2); bsr_free(&P->T);
  free(P->b); free(P->state); free(P->dirichlet); free(P->node_grid);
  free(P->face_geom); free(P->face_copies); free(P->aperture); free(P->pl);
  free(P->E_cell); free(P->Ebar_face); free(P->ups_face); free(P->rects); free(P->rects_q1);
  free(P->dk_face); free(P->dk_row); free(P->dk_col); free(P->dk_block); free(P->dk_comp); free(P->dk_val);
  memset(P, 0, sizeof(*P));
}

size_t fg_problem_size(void) { return sizeof(fg_problem); }
size_t fg_config_size(void) { return sizeof(fg_config); }
