/*
 * srfmg_oracle.c -- plain, slow FP64 CPU oracle for FAS full multigrid (FMG)
 * and segmental-refinement FAS-FMG (SR-FMG) on the cell-centred 7-point
 * Poisson problem on the unit cube with u = 0 on the boundary.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes, and where the paper defines it (Adams, Brown, Knepley,
 * Samtaney, "Segmental Refinement: A Multigrid Technique for Data Locality"):
 *   - grid and problem:        Sec. 2, Eq. (eq:eq), Eq. (eq:deq)
 *   - ghost-cell boundary:     Sec. 3.3 (linear interpolation of interior values)
 *   - FAS V-cycle FASMGV:      Sec. 3.1, Fig. "FAS multigrid V-cycle", Eq. (eq:cresid2)
 *   - full multigrid FMG:      Sec. 3.2, Fig. "Full multigrid"
 *   - SR regions and buffers:  Sec. 4, Eq. (eq:nb)
 *   - FASFMGSR / FASMGVSR:     Sec. 4, Figs. "FMG segmental refinement" and
 *                              "FAS V-cycle segmental refinement"
 *   - components:              Sec. 5.1 (piecewise-constant restriction,
 *                              linear prolongation, Chebyshev smoothers of
 *                              degree 2 (pre/post) and 1 (before each V-cycle))
 *
 * Readings taken where the paper is silent (each is also listed in the design
 * notes of the repository):
 *   - the operator is A = -Delta_h, (A u)_i = (6 u_i - sum of 6 neighbours)/h^2,
 *     so the solved system is A u = f with f = -Delta u (the paper writes L = Delta);
 *   - a ghost cell outside the domain holds minus its mirror interior cell
 *     (linear interpolation through u = 0 on the cell face); edge and corner
 *     ghosts apply the reflection once per outside dimension;
 *   - the smoother is Chebyshev iteration on D^-1 A with D = 6/h^2 over the
 *     interval [lo, hi] * lambda_max, lambda_max(D^-1 A) = 2; degree nu costs
 *     nu operator applications;
 *   - restriction of u and r: average of the 8 children; both prolongations
 *     (FMG and V-cycle correction): cell-centred trilinear, 1D weights 3/4, 1/4;
 *   - coarse right-hand sides f_k of FMG: 8-child average of f_{k+1};
 *   - coarsest solve: exact, by a banded Cholesky factorisation of the
 *     assembled coarsest-grid matrix (2^3 or 3^3 cells by default);
 *   - SR transition: each segment writes only its own genuine level-0 cells of
 *     the restricted solution and residual; the level-0 right-hand side is then
 *     formed globally;
 *   - on Omega^C_{k-1} \ Omega^F_{k-1} the coarse solution keeps the value it
 *     had at the end of the previous FMG stage.
 *
 * Index convention: a cell is (x, y, z) = (i, j, k); arrays are C-order
 * [z][y][x] with x fastest.  Level indices are global to the level grid.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXK 12
#define OR_MAXG 24

/* ------------------------------------------------------------------------ */
/* configuration (the library it is compared with has its own definition)    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n;            /* fine cells per unit length N = N_M (h = 1/N)           */
  int seg;          /* genuine segment edge on the finest level; 0 = plain FMG */
  int K;            /* number of SR levels                                     */
  int J[OR_MAXK];   /* J[k-1] = buffer width J_k, k = 1..K (Eq. eq:nb)         */
  int alpha, nu1, nu2;  /* F(alpha, nu1, nu2) cycle                            */
  double cheb_lo, cheb_hi;  /* Chebyshev interval, fractions of lambda_max     */
  int reverse_segments;     /* process segments in reverse order               */
  int n_threads;            /* OpenMP threads over segments (0: runtime default) */
  int n_coarse;             /* coarsest grid, cells per unit length; 0: 2 or 3 */
  int len[3];               /* domain [0,len0]x[0,len1]x[0,len2]; 0 reads as 1 */
  int stencil;              /* 7 (0 reads as 7) or 27                          */
  double w[3];              /* 27-point weights: faces, edges, corners         */
} or_config;

/* ------------------------------------------------------------------------ */
/* the operator A u = (1/h^2) (w0 u - w1 (sum of the 6 face neighbours)       */
/*   - w2 (sum of the 12 edge neighbours) - w3 (sum of the 8 corners)),       */
/* w0 = 6 w1 + 12 w2 + 8 w3; w1 = 1, w2 = w3 = 0 is the 7-point Laplacian of  */
/* Eq. (eq:deq); a 27-point stencil (Sec. 5.1) is consistent with -Delta when */
/* w1 + 4 w2 + 4 w3 = 1.  On the Fourier/sine mode with c_d = cos(theta_d)    */
/* A has the symbol (1/h^2)(w0 - 2 w1 sum c_d - 4 w2 sum_{d<e} c_d c_e        */
/* - 8 w3 c_0 c_1 c_2), multilinear in c, so its range over [-1, 1]^3 is      */
/* taken at the corners: lmax = the largest corner value / w0 bounds the      */
/* spectrum of D^-1 A, D = w0/h^2.                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  int pts;                  /* 7 or 27 */
  double w0, w1, w2, w3;
  double lmax;              /* sup of the spectrum of D^-1 A */
} Op;

static double op_symbol(const Op* o, const double c[3]) {
  return o->w0 - 2.0 * o->w1 * (c[0] + c[1] + c[2]) -
         4.0 * o->w2 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]) - 8.0 * o->w3 * c[0] * c[1] * c[2];
}

/* 0, or -2 if the stencil is not a consistent, positive definite one */
static int op_init(Op* o, int stencil, const double w[3]) {
  memset(o, 0, sizeof(*o));
  if (stencil == 0 || stencil == 7) {
    o->pts = 7;
    o->w1 = 1.0;
  } else if (stencil == 27) {
    o->pts = 27;
    o->w1 = w[0]; o->w2 = w[1]; o->w3 = w[2];
    if (fabs(o->w1 + 4.0 * o->w2 + 4.0 * o->w3 - 1.0) > 1e-12) return -2;
  } else {
    return -2;
  }
  o->w0 = 6.0 * o->w1 + 12.0 * o->w2 + 8.0 * o->w3;
  if (!(o->w0 > 0.0)) return -2;
  double top = 0.0;
  for (int v = 0; v < 8; ++v) {
    const double c[3] = {(v & 1) ? 1.0 : -1.0, (v & 2) ? 1.0 : -1.0, (v & 4) ? 1.0 : -1.0};
    const double s = op_symbol(o, c);
    if (v != 7 && !(s > 0.0)) return -2; /* only the constant mode may vanish */
    if (s > top) top = s;
  }
  o->lmax = top / o->w0;
  return 0;
}

/* domain lengths and operator of one problem */
typedef struct {
  int len[3];
  Op op;
} Geo;

static int geo_init(Geo* g, const or_config* c) {
  for (int d = 0; d < 3; ++d) {
    g->len[d] = c->len[d] ? c->len[d] : 1;
    if (g->len[d] < 1 || g->len[d] > 64) return -2;
  }
  return op_init(&g->op, c->stencil, c->w);
}

/* ------------------------------------------------------------------------ */
/* boxes: a block of cells [lo, hi) of a level grid plus a one-cell shell     */
/* ------------------------------------------------------------------------ */
typedef struct {
  const Geo* geo;        /* domain and operator */
  int n;                 /* cells per unit length of the level grid (h = 1/n) */
  int nd[3];             /* cells per dimension of the whole level grid, n len[d] */
  int lo[3], hi[3];      /* compute region */
  int ext[3];            /* stored extents hi - lo + 2 */
  long nstore;
} Box;

static void box_init(Box* b, const Geo* g, int n, const int lo[3], const int hi[3]) {
  b->geo = g;
  b->n = n;
  b->nstore = 1;
  for (int d = 0; d < 3; ++d) {
    b->nd[d] = n * g->len[d];
    b->lo[d] = lo[d];
    b->hi[d] = hi[d];
    b->ext[d] = hi[d] - lo[d] + 2;
    b->nstore *= b->ext[d];
  }
}

static void box_whole(Box* b, const Geo* g, int n) {
  int lo[3] = {0, 0, 0}, hi[3] = {n * g->len[0], n * g->len[1], n * g->len[2]};
  box_init(b, g, n, lo, hi);
}

/* storage offset of level cell (i, j, k); valid for lo-1 <= . <= hi */
static inline long at(const Box* b, int i, int j, int k) {
  return ((long)(k - b->lo[2] + 1) * b->ext[1] + (j - b->lo[1] + 1)) * b->ext[0] +
         (i - b->lo[0] + 1);
}

static double* zalloc(long n) { return (double*)calloc((size_t)n, sizeof(double)); }

/* ------------------------------------------------------------------------ */
/* boundary condition, Sec. 3.3: ghost cells outside the domain are set by    */
/* linear interpolation through u = 0 on the face, i.e. minus the mirror      */
/* interior value.  Passes run x, y, z over the full stored extent of the     */
/* other two dimensions, so edge and corner ghosts end with one sign flip per */
/* outside dimension.  Ghosts inside the domain (frozen SR ghosts) are kept.  */
/* ------------------------------------------------------------------------ */
static void fill_bc(const Box* b, double* a) {
  const int nx = b->nd[0], ny = b->nd[1], nz = b->nd[2];
  for (int k = b->lo[2] - 1; k <= b->hi[2]; ++k)
    for (int j = b->lo[1] - 1; j <= b->hi[1]; ++j) {
      if (b->lo[0] == 0) a[at(b, -1, j, k)] = -a[at(b, 0, j, k)];
      if (b->hi[0] == nx) a[at(b, nx, j, k)] = -a[at(b, nx - 1, j, k)];
    }
  for (int k = b->lo[2] - 1; k <= b->hi[2]; ++k)
    for (int i = b->lo[0] - 1; i <= b->hi[0]; ++i) {
      if (b->lo[1] == 0) a[at(b, i, -1, k)] = -a[at(b, i, 0, k)];
      if (b->hi[1] == ny) a[at(b, i, ny, k)] = -a[at(b, i, ny - 1, k)];
    }
  for (int j = b->lo[1] - 1; j <= b->hi[1]; ++j)
    for (int i = b->lo[0] - 1; i <= b->hi[0]; ++i) {
      if (b->lo[2] == 0) a[at(b, i, j, -1)] = -a[at(b, i, j, 0)];
      if (b->hi[2] == nz) a[at(b, i, j, nz)] = -a[at(b, i, j, nz - 1)];
    }
}

/* out = A u on the cells [rlo, rhi), 27-point operator; u must have valid
 * ghosts, edges and corners included */
static void apply_A27(const Box* b, const double* u, double* out, const int rlo[3],
                      const int rhi[3]) {
  const Op* o = &b->geo->op;
  const double ih2 = (double)b->n * (double)b->n;
  for (int k = rlo[2]; k < rhi[2]; ++k)
    for (int j = rlo[1]; j < rhi[1]; ++j)
      for (int i = rlo[0]; i < rhi[0]; ++i) {
        double sf = 0.0, se = 0.0, sc = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int far = (dx != 0) + (dy != 0) + (dz != 0);
              const double v = u[at(b, i + dx, j + dy, k + dz)];
              if (far == 1) sf += v;
              else if (far == 2) se += v;
              else if (far == 3) sc += v;
            }
        out[at(b, i, j, k)] =
            (o->w0 * u[at(b, i, j, k)] - o->w1 * sf - o->w2 * se - o->w3 * sc) * ih2;
      }
}

/* out = A u on the cells [rlo, rhi); u must have valid ghosts.  Eq. (eq:deq) */
static void apply_A(const Box* b, const double* u, double* out, const int rlo[3],
                    const int rhi[3]) {
  if (b->geo->op.pts == 27) {
    apply_A27(b, u, out, rlo, rhi);
    return;
  }
  const double ih2 = (double)b->n * (double)b->n; /* 1/h^2, h = 1/n */
  for (int k = rlo[2]; k < rhi[2]; ++k)
    for (int j = rlo[1]; j < rhi[1]; ++j)
      for (int i = rlo[0]; i < rhi[0]; ++i) {
        double nb = u[at(b, i - 1, j, k)] + u[at(b, i + 1, j, k)] + u[at(b, i, j - 1, k)] +
                    u[at(b, i, j + 1, k)] + u[at(b, i, j, k - 1)] + u[at(b, i, j, k + 1)];
        out[at(b, i, j, k)] = (6.0 * u[at(b, i, j, k)] - nb) * ih2;
      }
}

/* r = f - A u on the compute region of b (fill_bc applied to u first) */
static void residual(const Box* b, double* u, const double* f, double* r) {
  fill_bc(b, u);
  apply_A(b, u, r, b->lo, b->hi);
  for (int k = b->lo[2]; k < b->hi[2]; ++k)
    for (int j = b->lo[1]; j < b->hi[1]; ++j)
      for (int i = b->lo[0]; i < b->hi[0]; ++i) {
        long c = at(b, i, j, k);
        r[c] = f[c] - r[c];
      }
}

/* ------------------------------------------------------------------------ */
/* smoother S^nu(L, u, f) on the compute region of b (Sec. 5.1): Chebyshev    */
/* iteration for D^-1 A over [lo, hi], written as the textbook three-term     */
/* recurrence (theta = centre, delta = half width of the interval):           */
/*   r_0 = D^-1 (f - A x_0),  d_0 = r_0 / theta,  rho_0 = delta / theta        */
/*   x_{m+1} = x_m + d_m                                                       */
/*   r_{m+1} = D^-1 (f - A x_{m+1}),  rho_{m+1} = 1 / (2 theta/delta - rho_m)  */
/*   d_{m+1} = rho_{m+1} rho_m d_m + (2 rho_{m+1} / delta) r_{m+1}             */
/* Ghosts outside the domain are refreshed before every operator application; */
/* ghosts inside the domain stay frozen.                                       */
/* ------------------------------------------------------------------------ */
static void smooth(const Box* b, int nu, double cheb_lo, double cheb_hi, double* u,
                   const double* f, double* r, double* d) {
  if (nu <= 0) return;
  const Op* o = &b->geo->op;
  const double lmax = o->lmax; /* 2 for the 7-point operator */
  const double lo = cheb_lo * lmax, hi = cheb_hi * lmax;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const double dinv = 1.0 / (o->w0 * (double)b->n * (double)b->n); /* D^-1 = h^2/w0 */
  double rho_old = delta / theta;
  residual(b, u, f, r);
  for (int k = b->lo[2]; k < b->hi[2]; ++k)
    for (int j = b->lo[1]; j < b->hi[1]; ++j)
      for (int i = b->lo[0]; i < b->hi[0]; ++i) {
        long c = at(b, i, j, k);
        d[c] = dinv * r[c] / theta;
      }
  for (int m = 0; m < nu; ++m) {
    for (int k = b->lo[2]; k < b->hi[2]; ++k)
      for (int j = b->lo[1]; j < b->hi[1]; ++j)
        for (int i = b->lo[0]; i < b->hi[0]; ++i) {
          long c = at(b, i, j, k);
          u[c] += d[c];
        }
    if (m == nu - 1) break;
    residual(b, u, f, r);
    const double rho = 1.0 / (2.0 * theta / delta - rho_old);
    for (int k = b->lo[2]; k < b->hi[2]; ++k)
      for (int j = b->lo[1]; j < b->hi[1]; ++j)
        for (int i = b->lo[0]; i < b->hi[0]; ++i) {
          long c = at(b, i, j, k);
          d[c] = rho * rho_old * d[c] + (2.0 * rho / delta) * dinv * r[c];
        }
    rho_old = rho;
  }
}

/* ------------------------------------------------------------------------ */
/* restriction I^H_h and \hat I^H_h: average of the 8 children, on coarse     */
/* cells [rlo, rhi) (Sec. 5.1, "piecewise constant restriction")              */
/* ------------------------------------------------------------------------ */
static void restrict_avg(const Box* fb, const double* af, const Box* cb, double* ac,
                         const int rlo[3], const int rhi[3]) {
  for (int k = rlo[2]; k < rhi[2]; ++k)
    for (int j = rlo[1]; j < rhi[1]; ++j)
      for (int i = rlo[0]; i < rhi[0]; ++i) {
        double s = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) s += af[at(fb, 2 * i + a, 2 * j + b, 2 * k + c)];
        ac[at(cb, i, j, k)] = s / 8.0;
      }
}

/* ------------------------------------------------------------------------ */
/* prolongation I^h_H and Pi^h_H: cell-centred trilinear interpolation.       */
/* Fine cell i lies in coarse cell floor(i/2); its second coarse neighbour is */
/* on the side of the fine cell (i even: left, i odd: right); 1D weights 3/4  */
/* and 1/4.  Coarse ghosts must be valid.  add = 0 sets, add = 1 accumulates.  */
/* ------------------------------------------------------------------------ */
static int floordiv2(int i) { return (i >= 0) ? i / 2 : -((-i + 1) / 2); }

static void prolong(const Box* cb, const double* ac, const Box* fb, double* af,
                    const int rlo[3], const int rhi[3], int add) {
  for (int k = rlo[2]; k < rhi[2]; ++k)
    for (int j = rlo[1]; j < rhi[1]; ++j)
      for (int i = rlo[0]; i < rhi[0]; ++i) {
        const int f[3] = {i, j, k};
        int cc[3][2];
        double w[3][2];
        for (int d = 0; d < 3; ++d) {
          int c = floordiv2(f[d]);
          cc[d][0] = c;
          cc[d][1] = (f[d] - 2 * c == 0) ? c - 1 : c + 1;
          w[d][0] = 0.75;
          w[d][1] = 0.25;
        }
        double v = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
              v += w[0][a] * w[1][b] * w[2][c] * ac[at(cb, cc[0][a], cc[1][b], cc[2][c])];
        long o = at(fb, i, j, k);
        af[o] = add ? af[o] + v : v;
      }
}

/* the region C u G^SR of a box: compute region grown by one, clipped to the domain */
static void grown_region(const Box* b, int rlo[3], int rhi[3]) {
  for (int d = 0; d < 3; ++d) {
    rlo[d] = b->lo[d] > 0 ? b->lo[d] - 1 : 0;
    rhi[d] = b->hi[d] < b->nd[d] ? b->hi[d] + 1 : b->nd[d];
  }
}

/* ------------------------------------------------------------------------ */
/* coarsest-grid solve u = L_0^-1 f (Fig. "FAS multigrid V-cycle", else       */
/* branch).  The matrix is assembled column by column by applying the         */
/* operator to unit vectors; it is symmetric positive definite with nonzeros  */
/* only within |row - col| <= nx ny (7-point) or nx ny + nx + 1 (27-point),   */
/* so it is factored once by a Cholesky factorisation restricted to that band */
/* and solved by two triangular solves.                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int m, bw;      /* unknowns nx ny nz, half bandwidth */
  double* L;      /* m x m lower factor, entries within the band */
} Coarse;

static long cell_of(const Box* b, int q) {
  const int nx = b->nd[0], ny = b->nd[1];
  return at(b, q % nx, (q / nx) % ny, q / (nx * ny));
}

static int coarse_factor(Coarse* C, const Box* b) {
  const int nx = b->nd[0], ny = b->nd[1], nz = b->nd[2];
  const int m = nx * ny * nz;
  const int bw = (b->geo->op.pts == 27) ? nx * ny + nx + 1 : nx * ny;
  C->m = m; C->bw = bw;
  C->L = zalloc((long)m * m);
  double* e = zalloc(b->nstore);
  double* col = zalloc(b->nstore);
  if (!C->L || !e || !col) { free(e); free(col); return -3; }
  for (int q = 0; q < m; ++q) { /* column q of the operator */
    memset(e, 0, sizeof(double) * b->nstore);
    e[cell_of(b, q)] = 1.0;
    fill_bc(b, e);
    apply_A(b, e, col, b->lo, b->hi);
    for (int p = q; p < m && p <= q + bw; ++p) C->L[(long)p * m + q] = col[cell_of(b, p)];
  }
  free(e); free(col);
  for (int j = 0; j < m; ++j) { /* column-by-column Cholesky, A = L L^T */
    const int k0 = (j - bw > 0) ? j - bw : 0;
    double d = C->L[(long)j * m + j];
    for (int k = k0; k < j; ++k) d -= C->L[(long)j * m + k] * C->L[(long)j * m + k];
    if (!(d > 0.0)) return -1;
    d = sqrt(d);
    C->L[(long)j * m + j] = d;
    for (int i = j + 1; i < m && i <= j + bw; ++i) {
      double s = C->L[(long)i * m + j];
      const int kk = (i - bw > 0) ? i - bw : 0;
      for (int k = (kk > k0 ? kk : k0); k < j; ++k) s -= C->L[(long)i * m + k] * C->L[(long)j * m + k];
      C->L[(long)i * m + j] = s / d;
    }
  }
  return 0;
}

static void coarse_free(Coarse* C) { free(C->L); C->L = NULL; }

static void coarse_apply(const Coarse* C, const Box* b, double* u, const double* f) {
  const int m = C->m, bw = C->bw;
  double* x = zalloc(m);
  for (int p = 0; p < m; ++p) x[p] = f[cell_of(b, p)];
  for (int i = 0; i < m; ++i) { /* L y = f */
    double s = x[i];
    for (int k = (i - bw > 0 ? i - bw : 0); k < i; ++k) s -= C->L[(long)i * m + k] * x[k];
    x[i] = s / C->L[(long)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) { /* L^T u = y */
    double s = x[i];
    for (int k = i + 1; k < m && k <= i + bw; ++k) s -= C->L[(long)k * m + i] * x[k];
    x[i] = s / C->L[(long)i * m + i];
  }
  for (int p = 0; p < m; ++p) u[cell_of(b, p)] = x[p];
  free(x);
}

/* ------------------------------------------------------------------------ */
/* global (conventional) levels                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  Box box;
  double *u, *f, *rhs, *t, *r, *d, *rho, *e;
} GLevel;

typedef struct {
  or_config cfg;
  Geo geo;            /* domain and operator; every box points here */
  int G;              /* number of global levels; gl[G-1] is level 0 (transition / finest) */
  GLevel gl[OR_MAXG];
  Coarse coarse;      /* factor of the coarsest operator */
  int status;
} Solver;

static int glevel_alloc(GLevel* L, const Geo* g, int n) {
  box_whole(&L->box, g, n);
  long s = L->box.nstore;
  L->u = zalloc(s); L->f = zalloc(s); L->rhs = zalloc(s); L->t = zalloc(s);
  L->r = zalloc(s); L->d = zalloc(s); L->rho = zalloc(s); L->e = zalloc(s);
  return (L->u && L->f && L->rhs && L->t && L->r && L->d && L->rho && L->e) ? 0 : -1;
}

static void glevel_free(GLevel* L) {
  free(L->u); free(L->f); free(L->rhs); free(L->t);
  free(L->r); free(L->d); free(L->rho); free(L->e);
}

static void copy_store(const Box* b, double* dst, const double* src) {
  memcpy(dst, src, sizeof(double) * b->nstore);
}

/* FASMGV(L_k, u_k, f_k) on global level g (Fig. "FAS multigrid V-cycle");    */
/* u is gl[g].u, the right-hand side is rhs.                                   */
static void fasmgv(Solver* S, int g, const double* rhs) {
  GLevel* L = &S->gl[g];
  const or_config* c = &S->cfg;
  if (g == 0) {
    coarse_apply(&S->coarse, &L->box, L->u, rhs);
    return;
  }
  GLevel* C = &S->gl[g - 1];
  /* u_k <- S^nu1(L_k, u_k, f_k) */
  smooth(&L->box, c->nu1, c->cheb_lo, c->cheb_hi, L->u, rhs, L->r, L->d);
  /* r_k <- f_k - L_k u_k */
  residual(&L->box, L->u, rhs, L->r);
  /* u_{k-1} <- \hat I u_k ; r_{k-1} <- I r_k */
  restrict_avg(&L->box, L->u, &C->box, C->u, C->box.lo, C->box.hi);
  restrict_avg(&L->box, L->r, &C->box, C->rho, C->box.lo, C->box.hi);
  /* t_{k-1} <- u_{k-1} */
  fill_bc(&C->box, C->u);
  copy_store(&C->box, C->t, C->u);
  /* w_{k-1} <- FASMGV(L_{k-1}, u_{k-1}, r_{k-1} + L_{k-1} u_{k-1})  (Eq. eq:cresid2) */
  apply_A(&C->box, C->u, C->rhs, C->box.lo, C->box.hi);
  for (long q = 0; q < C->box.nstore; ++q) C->rhs[q] += C->rho[q];
  fasmgv(S, g - 1, C->rhs);
  /* u_k <- u_k + I(w_{k-1} - t_{k-1}) */
  for (long q = 0; q < C->box.nstore; ++q) C->e[q] = C->u[q] - C->t[q];
  fill_bc(&C->box, C->e);
  prolong(&C->box, C->e, &L->box, L->u, L->box.lo, L->box.hi, 1);
  /* u_k <- S^nu2(L_k, u_k, f_k) */
  smooth(&L->box, c->nu2, c->cheb_lo, c->cheb_hi, L->u, rhs, L->r, L->d);
}

/* FMG (Fig. "Full multigrid") over global levels 0..gtop, f in gl[.].f */
static void fmg_global(Solver* S, int gtop) {
  const or_config* c = &S->cfg;
  GLevel* L0 = &S->gl[0];
  memset(L0->u, 0, sizeof(double) * L0->box.nstore);
  fasmgv(S, 0, L0->f);
  for (int g = 1; g <= gtop; ++g) {
    GLevel* L = &S->gl[g];
    GLevel* C = &S->gl[g - 1];
    fill_bc(&C->box, C->u);
    prolong(&C->box, C->u, &L->box, L->u, L->box.lo, L->box.hi, 0); /* u_k <- Pi u_{k-1} */
    smooth(&L->box, c->alpha, c->cheb_lo, c->cheb_hi, L->u, L->f, L->r, L->d); /* S^alpha */
    fasmgv(S, g, L->f);
  }
}

/* ------------------------------------------------------------------------ */
/* segmental refinement (Sec. 4)                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  Box box[OR_MAXK + 1];                 /* box[k]: compute region Omega^C_k, k = 1..K */
  double *u[OR_MAXK + 1], *t[OR_MAXK + 1], *rhs[OR_MAXK + 1];
  int g0lo[3], g0hi[3];                 /* genuine region on level 0 */
} Segment;

typedef struct {
  double *r, *d, *rho, *e;
} Scratch;

typedef struct {
  int K, nsd[3], nseg;                  /* segments per dimension, total */
  int nk[OR_MAXK + 1];                  /* level sizes N_k, k = 0..K */
  double* fk[OR_MAXK + 1];              /* f_k on SR levels (global arrays of the level grid) */
  Box fbox[OR_MAXK + 1];
  Segment* seg;
} SR;

/* segment p's compute region on SR level k: genuine region grown by J_k and
 * clipped by the domain, Omega^C_k = Omega^{V+J_k} cap Omega_k (Sec. 4) */
static void seg_coords(const SR* R, int p, int q[3]) {
  q[0] = p % R->nsd[0];
  q[1] = (p / R->nsd[0]) % R->nsd[1];
  q[2] = p / (R->nsd[0] * R->nsd[1]);
}

static void seg_box(const Solver* S, const SR* R, int p, int k, Box* b) {
  const or_config* c = &S->cfg;
  const int sk = c->seg >> (R->K - k); /* genuine edge on level k */
  int q[3];
  seg_coords(R, p, q);
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    const int nd = R->nk[k] * S->geo.len[d];
    lo[d] = q[d] * sk - c->J[k - 1];
    hi[d] = (q[d] + 1) * sk + c->J[k - 1];
    if (lo[d] < 0) lo[d] = 0;
    if (hi[d] > nd) hi[d] = nd;
  }
  box_init(b, &S->geo, R->nk[k], lo, hi);
}

/* one FMG stage k for segment P, up to and including the level-1 restriction:
 * Pi onto C u G^SR, S^alpha, then the down-leg of FASMGVSR(k) (Fig. "FAS
 * V-cycle segmental refinement"), restriction to level 0 written for the
 * segment's own genuine cells. */
static void sr_down(Solver* S, SR* R, Segment* P, int k, Scratch* w) {
  const or_config* c = &S->cfg;
  GLevel* L0 = &S->gl[S->G - 1];
  int rlo[3], rhi[3];
  /* u_k <- Pi^k_{k-1} u_{k-1} on Omega^C_k u Omega^GSR_k */
  {
    const Box* cb = (k == 1) ? &L0->box : &P->box[k - 1];
    const double* cu = (k == 1) ? L0->u : P->u[k - 1];
    if (k > 1) fill_bc(&P->box[k - 1], P->u[k - 1]);
    grown_region(&P->box[k], rlo, rhi);
    prolong(cb, cu, &P->box[k], P->u[k], rlo, rhi, 0);
  }
  /* the level's right-hand side for this stage is f_k */
  {
    const Box* b = &P->box[k];
    for (int z = b->lo[2]; z < b->hi[2]; ++z)
      for (int y = b->lo[1]; y < b->hi[1]; ++y)
        for (int x = b->lo[0]; x < b->hi[0]; ++x)
          P->rhs[k][at(b, x, y, z)] = R->fk[k][at(&R->fbox[k], x, y, z)];
  }
  /* u_k <- S^alpha(L_k, u_k, f_k) on Omega^C_k */
  smooth(&P->box[k], c->alpha, c->cheb_lo, c->cheb_hi, P->u[k], P->rhs[k], w->r, w->d);
  /* FASMGVSR(L_k, u_k, f_k): down-leg over levels k..1 */
  for (int j = k; j >= 1; --j) {
    const Box* b = &P->box[j];
    smooth(b, c->nu1, c->cheb_lo, c->cheb_hi, P->u[j], P->rhs[j], w->r, w->d);
    residual(b, P->u[j], P->rhs[j], w->r); /* r_j - L_j u_j on Omega^C_j */
    if (j > 1) {
      const Box* cb = &P->box[j - 1];
      int flo[3], fhi[3]; /* Omega^F: the level-(j-1) cells under Omega^C_j */
      for (int d = 0; d < 3; ++d) { flo[d] = b->lo[d] / 2; fhi[d] = b->hi[d] / 2; }
      /* u_{j-1} <- \hat I u_j on Omega^F */
      restrict_avg(b, P->u[j], cb, P->u[j - 1], flo, fhi);
      /* t_{j-1} <- u_{j-1} */
      fill_bc(cb, P->u[j - 1]);
      copy_store(cb, P->t[j - 1], P->u[j - 1]);
      /* r_{j-1} <- I(r_j - L_j u_j) + L_{j-1} u_{j-1} on Omega^F,
       * r_{j-1} <- L_{j-1} u_{j-1} on Omega^C \ Omega^F */
      memset(w->rho, 0, sizeof(double) * cb->nstore);
      restrict_avg(b, w->r, cb, w->rho, flo, fhi);
      apply_A(cb, P->u[j - 1], P->rhs[j - 1], cb->lo, cb->hi);
      for (int z = flo[2]; z < fhi[2]; ++z)
        for (int y = flo[1]; y < fhi[1]; ++y)
          for (int x = flo[0]; x < fhi[0]; ++x) P->rhs[j - 1][at(cb, x, y, z)] += w->rho[at(cb, x, y, z)];
    } else {
      /* transition: this segment's genuine level-0 cells of \hat I u_1 and
       * I(r_1 - L_1 u_1).  \hat I u_1 goes to t_0, not u_0: segments that have
       * not yet prolongated in this stage still read u_0 from the previous stage. */
      restrict_avg(b, P->u[1], &L0->box, L0->t, P->g0lo, P->g0hi);
      restrict_avg(b, w->r, &L0->box, L0->rho, P->g0lo, P->g0hi);
    }
  }
}

/* the up-leg of FASMGVSR(k) for segment P: corrections u_j += I(w_{j-1} - t_{j-1})
 * on Omega^C_j u Omega^GSR_j followed by S^nu2 on Omega^C_j, j = 1..k */
static void sr_up(Solver* S, SR* R, Segment* P, int k, Scratch* w) {
  const or_config* c = &S->cfg;
  GLevel* L0 = &S->gl[S->G - 1];
  (void)R;
  int rlo[3], rhi[3];
  for (int j = 1; j <= k; ++j) {
    const Box* cb;
    const double* e;
    if (j == 1) {
      cb = &L0->box;
      e = L0->e; /* w_0 - t_0, boundary ghosts already filled */
    } else {
      cb = &P->box[j - 1];
      for (long q = 0; q < cb->nstore; ++q) w->e[q] = P->u[j - 1][q] - P->t[j - 1][q];
      fill_bc(cb, w->e);
      e = w->e;
    }
    grown_region(&P->box[j], rlo, rhi);
    prolong(cb, e, &P->box[j], P->u[j], rlo, rhi, 1);
    smooth(&P->box[j], c->nu2, c->cheb_lo, c->cheb_hi, P->u[j], P->rhs[j], w->r, w->d);
  }
}

/* ------------------------------------------------------------------------ */
/* public entry points                                                        */
/* ------------------------------------------------------------------------ */

/* halvings from an n^3 grid down to the coarsest grid: nc cells, or 2 or 3
 * cells when nc == 0; -1 if n does not coarsen to it */
static int levels_below(int n, int nc) {
  int m = 0;
  while (nc ? n > nc : n > 3) {
    if (n % 2) return -1;
    n /= 2;
    ++m;
  }
  if (nc) return (n == nc) ? m : -1;
  return (n >= 2) ? m : -1;
}

static void load_grid(const Box* b, double* a, const double* src) {
  const int nx = b->nd[0], ny = b->nd[1], nz = b->nd[2];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) a[at(b, i, j, k)] = src[((long)k * ny + j) * nx + i];
}

static void store_grid(const Box* b, const double* a, double* dst) {
  const int nx = b->nd[0], ny = b->nd[1], nz = b->nd[2];
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) dst[((long)k * ny + j) * nx + i] = a[at(b, i, j, k)];
}

/* validation shared by the solvers; returns 0 if the configuration is usable */
int or_check_config(const or_config* c) {
  Geo g;
  if (geo_init(&g, c)) return -2;
  if (c->n_coarse < 0 || c->n_coarse > 16) return -2;
  if (c->n < 1 || levels_below(c->n, c->n_coarse) < 0) return -2;
  if (c->alpha < 0 || c->nu1 < 0 || c->nu2 < 0) return -2;
  if (!(c->cheb_lo > 0.0 && c->cheb_hi > c->cheb_lo)) return -2;
  if (c->seg == 0 || c->K == 0) return 0;
  if (c->K < 0 || c->K > OR_MAXK || c->seg < 0) return -2;
  if (c->n % c->seg) return -2; /* whole segments per unit length */
  if (c->seg % (1 << c->K)) return -2;
  const int n0 = c->n >> c->K;
  if (levels_below(n0, c->n_coarse) < 0) return -2;
  for (int k = 1; k <= c->K; ++k) {
    if (c->J[k - 1] < 0 || c->J[k - 1] % 2) return -2;
    if (k >= 2 && 2 * c->J[k - 2] < c->J[k - 1]) return -2; /* coarse box covers prolongation */
  }
  return 0;
}

/* Buffer schedule Eq. (eq:nb): J_k = 2 floor((A + B (K - k)) / 2), k = 1..K */
void or_buffer_schedule(int A, int B, int K, int* J) {
  for (int k = 1; k <= K; ++k) {
    int v = A + B * (K - k);
    J[k - 1] = 2 * (v / 2);
  }
}

static int solver_init(Solver* S, const or_config* c, int n_global_top) {
  memset(S, 0, sizeof(*S));
  S->cfg = *c;
  if (geo_init(&S->geo, c)) return -2;
  int m = levels_below(n_global_top, c->n_coarse);
  S->G = m + 1;
  if (m < 0 || S->G > OR_MAXG) return -2;
  for (int g = 0; g < S->G; ++g)
    if (glevel_alloc(&S->gl[g], &S->geo, n_global_top >> (S->G - 1 - g))) return -3;
  return coarse_factor(&S->coarse, &S->gl[0].box);
}

static void solver_free(Solver* S) {
  for (int g = 0; g < S->G; ++g) glevel_free(&S->gl[g]);
  coarse_free(&S->coarse);
}

/* restrict f down the global levels: f_{k-1} = average of f_k */
static void global_f_hierarchy(Solver* S) {
  for (int g = S->G - 1; g >= 1; --g)
    restrict_avg(&S->gl[g].box, S->gl[g].f, &S->gl[g - 1].box, S->gl[g - 1].f,
                 S->gl[g - 1].box.lo, S->gl[g - 1].box.hi);
}

static int solve_plain(const or_config* c, const double* f, double* u) {
  Solver S;
  int st = solver_init(&S, c, c->n);
  if (st) { solver_free(&S); return st; }
  load_grid(&S.gl[S.G - 1].box, S.gl[S.G - 1].f, f);
  global_f_hierarchy(&S);
  fmg_global(&S, S.G - 1);
  store_grid(&S.gl[S.G - 1].box, S.gl[S.G - 1].u, u);
  st = S.status;
  solver_free(&S);
  return st;
}

static int solve_sr(const or_config* c, const double* f, double* u) {
  const int K = c->K;
  SR R;
  memset(&R, 0, sizeof(R));
  R.K = K;
  for (int k = 0; k <= K; ++k) R.nk[k] = c->n >> (K - k);
  Solver S;
  int st = solver_init(&S, c, R.nk[0]);
  if (st) { solver_free(&S); return st; }
  R.nseg = 1;
  for (int d = 0; d < 3; ++d) {
    R.nsd[d] = c->n * S.geo.len[d] / c->seg;
    R.nseg *= R.nsd[d];
  }
  /* f_k on all SR levels, restricted down from f_K, then down the global levels */
  for (int k = 1; k <= K; ++k) {
    box_whole(&R.fbox[k], &S.geo, R.nk[k]);
    R.fk[k] = zalloc(R.fbox[k].nstore);
    if (!R.fk[k]) st = -3;
  }
  R.seg = (Segment*)calloc((size_t)R.nseg, sizeof(Segment));
  if (!R.seg) st = -3;
  if (st) goto done;
  load_grid(&R.fbox[K], R.fk[K], f);
  for (int k = K; k >= 2; --k)
    restrict_avg(&R.fbox[k], R.fk[k], &R.fbox[k - 1], R.fk[k - 1], R.fbox[k - 1].lo,
                 R.fbox[k - 1].hi);
  {
    GLevel* L0 = &S.gl[S.G - 1];
    restrict_avg(&R.fbox[1], R.fk[1], &L0->box, L0->f, L0->box.lo, L0->box.hi);
  }
  global_f_hierarchy(&S);
  long maxstore = 0;
  for (int p = 0; p < R.nseg; ++p) {
    Segment* P = &R.seg[p];
    const int s0 = c->seg >> K;
    int q[3];
    seg_coords(&R, p, q);
    for (int d = 0; d < 3; ++d) { P->g0lo[d] = q[d] * s0; P->g0hi[d] = (q[d] + 1) * s0; }
    for (int k = 1; k <= K; ++k) {
      seg_box(&S, &R, p, k, &P->box[k]);
      long s = P->box[k].nstore;
      if (s > maxstore) maxstore = s;
      P->u[k] = zalloc(s);
      P->t[k] = zalloc(s);
      P->rhs[k] = zalloc(s);
      if (!P->u[k] || !P->t[k] || !P->rhs[k]) st = -3;
    }
  }
  if (st) goto done;
  {
    int nth = 1;
#ifdef _OPENMP
    nth = (c->n_threads > 0) ? c->n_threads : omp_get_max_threads();
#endif
    Scratch* W = (Scratch*)calloc((size_t)nth, sizeof(Scratch));
    if (!W) { st = -3; goto done; }
    for (int t = 0; t < nth; ++t) {
      W[t].r = zalloc(maxstore); W[t].d = zalloc(maxstore);
      W[t].rho = zalloc(maxstore); W[t].e = zalloc(maxstore);
      if (!W[t].r || !W[t].d || !W[t].rho || !W[t].e) st = -3;
    }
    if (!st) {
      GLevel* L0 = &S.gl[S.G - 1];
      /* u_0 <- FMG (conventional solver up to the transition level) */
      fmg_global(&S, S.G - 1);
      for (int k = 1; k <= K; ++k) {
        fill_bc(&L0->box, L0->u);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
        for (int it = 0; it < R.nseg; ++it) {
          int tid = 0;
#ifdef _OPENMP
          tid = omp_get_thread_num();
#endif
          int p = c->reverse_segments ? R.nseg - 1 - it : it;
          sr_down(&S, &R, &R.seg[p], k, &W[tid]);
        }
        /* level 0: u_0 <- \hat I u_1 (owner-written into t_0), t_0 <- u_0,
         * r_0 <- rho_0 + L_0 u_0, w_0 <- FASMGV(L_0, u_0, r_0) */
        copy_store(&L0->box, L0->u, L0->t);
        fill_bc(&L0->box, L0->u);
        copy_store(&L0->box, L0->t, L0->u);
        apply_A(&L0->box, L0->u, L0->rhs, L0->box.lo, L0->box.hi);
        for (long q = 0; q < L0->box.nstore; ++q) L0->rhs[q] += L0->rho[q];
        fasmgv(&S, S.G - 1, L0->rhs);
        for (long q = 0; q < L0->box.nstore; ++q) L0->e[q] = L0->u[q] - L0->t[q];
        fill_bc(&L0->box, L0->e);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
#endif
        for (int it = 0; it < R.nseg; ++it) {
          int tid = 0;
#ifdef _OPENMP
          tid = omp_get_thread_num();
#endif
          int p = c->reverse_segments ? R.nseg - 1 - it : it;
          sr_up(&S, &R, &R.seg[p], k, &W[tid]);
        }
      }
      /* return u_K: the genuine cells of every segment */
      const int nx = R.fbox[K].nd[0], ny = R.fbox[K].nd[1];
      for (int p = 0; p < R.nseg; ++p) {
        Segment* P = &R.seg[p];
        const Box* b = &P->box[K];
        const int sK = c->seg;
        int q[3];
        seg_coords(&R, p, q);
        for (int z = q[2] * sK; z < (q[2] + 1) * sK; ++z)
          for (int y = q[1] * sK; y < (q[1] + 1) * sK; ++y)
            for (int x = q[0] * sK; x < (q[0] + 1) * sK; ++x)
              u[((long)z * ny + y) * nx + x] = P->u[K][at(b, x, y, z)];
      }
      st = S.status;
    }
    for (int t = 0; t < nth; ++t) { free(W[t].r); free(W[t].d); free(W[t].rho); free(W[t].e); }
    free(W);
  }
done:
  if (R.seg)
    for (int p = 0; p < R.nseg; ++p)
      for (int k = 1; k <= K; ++k) { free(R.seg[p].u[k]); free(R.seg[p].t[k]); free(R.seg[p].rhs[k]); }
  free(R.seg);
  for (int k = 1; k <= K; ++k) free(R.fk[k]);
  solver_free(&S);
  return st;
}

/* FMG (seg == 0 or K == 0) or SR-FMG (FASFMGSR) on f (n^3, C order); u = result */
int or_solve(const or_config* c, const double* f, double* u) {
  int st = or_check_config(c);
  if (st) return st;
  if (c->seg == 0 || c->K == 0) return solve_plain(c, f, u);
  return solve_sr(c, f, u);
}

/* one FAS V-cycle FASMGV on the global n^3 grid; u is updated in place */
int or_vcycle(const or_config* c, const double* f, double* u) {
  or_config pc = *c;
  pc.seg = 0;
  pc.K = 0;
  int st = or_check_config(&pc);
  if (st) return st;
  Solver S;
  st = solver_init(&S, &pc, c->n);
  if (!st) {
    GLevel* L = &S.gl[S.G - 1];
    load_grid(&L->box, L->f, f);
    load_grid(&L->box, L->u, u);
    fasmgv(&S, S.G - 1, L->f);
    store_grid(&L->box, L->u, u);
    st = S.status;
  }
  solver_free(&S);
  return st;
}

/* max |f - A u| over the n^3 cells of global level L (uses L->r) */
static double residual_max(GLevel* L, const double* f) {
  const Box* b = &L->box;
  residual(b, L->u, f, L->r);
  double m = 0.0;
  for (int k = 0; k < b->nd[2]; ++k)
    for (int j = 0; j < b->nd[1]; ++j)
      for (int i = 0; i < b->nd[0]; ++i) {
        const double v = fabs(L->r[at(b, i, j, k)]);
        if (!(v <= m)) m = v; /* a NaN sticks */
      }
  return m;
}

/* Iterative V-cycle solver (the comparison solver of Sec. 5.3, Fig. "Errors
 * of all solvers"): starting from the u passed in, apply FASMGV on the
 * global grid until ||f - A u||_inf <= rtol ||f||_inf or max_cycles cycles
 * have run.  *cycles = V-cycles applied, *rel = final ||f - A u|| / ||f||
 * (0 when both norms are 0).  Returns 0, or -6 if a residual is not finite. */
int or_vsolve(const or_config* c, const double* f, double* u, double rtol, int max_cycles,
              int* cycles, double* rel) {
  or_config pc = *c;
  pc.seg = 0;
  pc.K = 0;
  int st = or_check_config(&pc);
  if (st) return st;
  if (max_cycles < 0 || !(rtol >= 0.0)) return -1;
  Solver S;
  st = solver_init(&S, &pc, c->n);
  if (!st) {
    GLevel* L = &S.gl[S.G - 1];
    const long cells = (long)L->box.nd[0] * L->box.nd[1] * L->box.nd[2];
    double fnorm = 0.0;
    for (long q = 0; q < cells; ++q)
      if (!(fabs(f[q]) <= fnorm)) fnorm = fabs(f[q]);
    load_grid(&L->box, L->f, f);
    load_grid(&L->box, L->u, u);
    int it = 0;
    double r = residual_max(L, L->f);
    for (;;) {
      const double q = (fnorm > 0.0) ? r / fnorm : (r > 0.0 ? INFINITY : 0.0);
      *rel = q;
      if (!isfinite(r)) { st = -6; break; }
      if (q <= rtol || it >= max_cycles) break;
      fasmgv(&S, S.G - 1, L->f);
      ++it;
      r = residual_max(L, L->f);
    }
    *cycles = it;
    store_grid(&L->box, L->u, u);
    if (!st) st = S.status;
  }
  solver_free(&S);
  return st;
}

/* ---- single components on a whole grid (unpadded C-order arrays) --------
 * The *_g entry points take the grid (n cells per unit length, the domain
 * lengths len) and the operator (stencil, w) from a configuration; the plain
 * ones are the unit cube with the 7-point operator. */

static or_config cube7(int n) {
  or_config c;
  memset(&c, 0, sizeof(c));
  c.n = n;
  return c;
}

int or_apply_g(const or_config* c, const double* u, double* out) {
  Geo g;
  if (c->n < 1 || geo_init(&g, c)) return -2;
  Box b;
  box_whole(&b, &g, c->n);
  double* a = zalloc(b.nstore);
  double* o = zalloc(b.nstore);
  if (!a || !o) { free(a); free(o); return -3; }
  load_grid(&b, a, u);
  fill_bc(&b, a);
  apply_A(&b, a, o, b.lo, b.hi);
  store_grid(&b, o, out);
  free(a); free(o);
  return 0;
}

int or_smooth_g(const or_config* c, int nu, const double* f, double* u) {
  Geo g;
  if (c->n < 1 || geo_init(&g, c)) return -2;
  Box b;
  box_whole(&b, &g, c->n);
  double *a = zalloc(b.nstore), *ff = zalloc(b.nstore), *r = zalloc(b.nstore), *d = zalloc(b.nstore);
  if (!a || !ff || !r || !d) { free(a); free(ff); free(r); free(d); return -3; }
  load_grid(&b, a, u);
  load_grid(&b, ff, f);
  smooth(&b, nu, c->cheb_lo, c->cheb_hi, a, ff, r, d);
  store_grid(&b, a, u);
  free(a); free(ff); free(r); free(d);
  return 0;
}

int or_residual_g(const or_config* c, const double* f, const double* u, double* r) {
  Geo g;
  if (c->n < 1 || geo_init(&g, c)) return -2;
  Box b;
  box_whole(&b, &g, c->n);
  double *a = zalloc(b.nstore), *ff = zalloc(b.nstore), *rr = zalloc(b.nstore);
  if (!a || !ff || !rr) { free(a); free(ff); free(rr); return -3; }
  load_grid(&b, a, u);
  load_grid(&b, ff, f);
  residual(&b, a, ff, rr);
  store_grid(&b, rr, r);
  free(a); free(ff); free(rr);
  return 0;
}

/* c describes the fine grid (c->n even) */
int or_restrict_g(const or_config* c, const double* a, double* ac) {
  Geo g;
  if (c->n < 2 || c->n % 2 || geo_init(&g, c)) return -2;
  Box fb, cb;
  box_whole(&fb, &g, c->n);
  box_whole(&cb, &g, c->n / 2);
  double *x = zalloc(fb.nstore), *y = zalloc(cb.nstore);
  if (!x || !y) { free(x); free(y); return -3; }
  load_grid(&fb, x, a);
  restrict_avg(&fb, x, &cb, y, cb.lo, cb.hi);
  store_grid(&cb, y, ac);
  free(x); free(y);
  return 0;
}

/* fine grid (2 n per unit length) = trilinear prolongation of the coarse grid
 * c describes (boundary ghosts by Sec. 3.3) */
int or_prolong_g(const or_config* c, const double* ac, double* af) {
  Geo g;
  if (c->n < 1 || geo_init(&g, c)) return -2;
  Box fb, cb;
  box_whole(&cb, &g, c->n);
  box_whole(&fb, &g, 2 * c->n);
  double *x = zalloc(cb.nstore), *y = zalloc(fb.nstore);
  if (!x || !y) { free(x); free(y); return -3; }
  load_grid(&cb, x, ac);
  fill_bc(&cb, x);
  prolong(&cb, x, &fb, y, fb.lo, fb.hi, 0);
  store_grid(&fb, y, af);
  free(x); free(y);
  return 0;
}

int or_coarse_solve_g(const or_config* c, const double* f, double* u) {
  Geo g;
  if (c->n < 1 || geo_init(&g, c)) return -2;
  Box b;
  box_whole(&b, &g, c->n);
  double *ff = zalloc(b.nstore), *uu = zalloc(b.nstore);
  Coarse C;
  memset(&C, 0, sizeof(C));
  int st = (ff && uu) ? coarse_factor(&C, &b) : -3;
  if (!st) {
    load_grid(&b, ff, f);
    coarse_apply(&C, &b, uu, ff);
    store_grid(&b, uu, u);
  }
  coarse_free(&C);
  free(ff); free(uu);
  return st;
}

int or_apply(int n, const double* u, double* out) {
  const or_config c = cube7(n);
  return or_apply_g(&c, u, out);
}

int or_smooth(int n, int nu, double cheb_lo, double cheb_hi, const double* f, double* u) {
  or_config c = cube7(n);
  c.cheb_lo = cheb_lo;
  c.cheb_hi = cheb_hi;
  return or_smooth_g(&c, nu, f, u);
}

int or_residual(int n, const double* f, const double* u, double* r) {
  const or_config c = cube7(n);
  return or_residual_g(&c, f, u, r);
}

int or_restrict(int n, const double* a, double* ac) {
  const or_config c = cube7(n);
  return or_restrict_g(&c, a, ac);
}

int or_prolong(int nc, const double* ac, double* af) {
  const or_config c = cube7(nc);
  return or_prolong_g(&c, ac, af);
}

int or_coarse_solve(int n, const double* f, double* u) {
  const or_config c = cube7(n);
  return or_coarse_solve_g(&c, f, u);
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
