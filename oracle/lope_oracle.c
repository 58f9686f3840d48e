/*
 * FP64 reference ("oracle") for the locally-oriented (LOPe) stencil hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is built into oracle/liboracle.so and is
 * used by the tests, by the smoke check and by the benchmark's CPU baseline.
 * The library path (paper_1502_03504_gb300/) never links, loads or calls it,
 * and it shares no code with the CUDA kernels.
 *
 * What it computes (Rasmussen et al., "Locally-Oriented Programming", arXiv
 * 1502.03504):
 *  - A local function writes only the local element U(0,0) and reads an
 *    immutable halo U(dx,dy) around it (Sec. 2, Sec. 2.2 "Concurrent
 *    functions", Fig. 1).  Offsets follow the paper's zero-based local index
 *    notation (Sec. 2.2 "LOPe index notation"): the first offset runs
 *    left/right, the second below/above.  Here the first offset (dx) runs
 *    along the fastest, contiguous axis, the second (dy) along the next one and
 *    a third (dz) along the slowest axis of a 3D grid.
 *  - The function is applied at every interior point from a frozen snapshot of
 *    the state at the time of invocation (Sec. 2.2 on double buffering; Sec.
 *    3.5, the implicit-synchronisation constraint), i.e. Jacobi semantics.
 *  - The halo holds boundary-value information (Sec. 2.2 "Halo regions"); the
 *    cyclic boundary of Sec. 3.2 (HALO_TRANSFER(U, BC=CYCLIC)) is a periodic
 *    wrap; a Dirichlet boundary holds a fixed value in the halo.  The halo is
 *    refreshed after every sweep (Sec. 3.2), so each step reads ghosts built
 *    from the current state.
 *  - The "serial execution by inlining" target of Sec. 4.1 is what this file
 *    is: a plain loop over every element calling the local function.
 *
 * Adjoint: u_{t+1} = A u_t for the linear stencils.  The discrete adjoint
 * lambda_t = A^T lambda_{t+1} is computed here by scattering each point's
 * weights onto its neighbours (the transpose written out), not by reusing the
 * forward gather.  The full trajectory is stored; no checkpointing.
 *
 * Everything is IEEE binary64 with round-to-nearest; build with
 * -ffp-contract=off so that x86 and Arm give identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_PERIODIC = 0, OR_DIRICHLET = 1 };

/* Local-function kinds (same numbering as the library's builtin names). */
enum {
  OR_LINEAR = 0,   /* general linear box stencil from a weight table          */
  OR_JACOBI5 = 1,  /* 2D: u + c (E + W + N + S - 4u)                          */
  OR_DIFF7 = 2,    /* 3D: u + c (sum of 6 face neighbours - 6u)               */
  OR_STAR9R2 = 3,  /* 2D: u + c (L4x u + L4y u), 4th-order 1D Laplacians      */
  OR_SWE = 4,      /* 2D, 3 fields (h,u,v): linearised C-grid shallow water   */
  OR_SWEFLUX = 5,  /* 2D, 3 fields (eta,u,v): nonlinear flux-form C-grid SWE  */
  OR_USER = 6      /* a user-written local function (see oracle_apply_user)   */
};

enum { OR_OK = 0, OR_ERR = 1 };

#define OR_MAXF 3

typedef struct {
  int ndim;
  int64_t n[3];       /* extents, slowest..fastest; n[0] = 1 for 2D grids      */
  int bc[3][2];       /* per axis (slowest..fastest), per side (low, high)    */
  double bval[3][2];  /* Dirichlet values                                     */
} or_grid;

typedef struct {
  const or_grid* g;
  const double* f[OR_MAXF]; /* frozen snapshot of each field                  */
  int64_t p[3];             /* the local element                              */
} or_acc;

/* A user-written local function: reads taps through U(acc, f, dx, dy, dz) and
 * writes out[f]; P holds its parameters. */
typedef double (*or_tap_fn)(const void* acc, int f, int dx, int dy, int dz);
typedef void (*or_user_fn)(const void* acc, or_tap_fn U, const double* P, double* out);

typedef struct {
  int kind;
  int radius;             /* for OR_LINEAR                                    */
  or_user_fn user;        /* for OR_USER                                      */
  int user_nf;            /* for OR_USER                                      */
  const double* prm;      /* c, or (dt, g, H) for OR_SWE, (dt, g, f, H) for OR_SWEFLUX */
  const double* w;        /* OR_LINEAR weights, (2r+1)^ndim, slowest first    */
} or_stencil;

static int64_t npoints(const or_grid* g) { return g->n[0] * g->n[1] * g->n[2]; }

/* U(dx,dy,dz) of field k: the local element plus offset, with the halo value
 * when the offset leaves the domain.  A Dirichlet side returns its fixed value;
 * periodic axes wrap (Sec. 3.2, U(M+1,:) = U(1,:) of the right-hand neighbour,
 * which on a single image is the cyclic wrap). */
static double U(const or_acc* a, int k, int dx, int dy, int dz) {
  const or_grid* g = a->g;
  int64_t q[3] = {a->p[0] + dz, a->p[1] + dy, a->p[2] + dx};
  for (int ax = 0; ax < 3; ax++) {
    if (q[ax] < 0 && g->bc[ax][0] == OR_DIRICHLET) return g->bval[ax][0];
    if (q[ax] >= g->n[ax] && g->bc[ax][1] == OR_DIRICHLET) return g->bval[ax][1];
  }
  for (int ax = 0; ax < 3; ax++) {
    int64_t m = g->n[ax];
    q[ax] = ((q[ax] % m) + m) % m;
  }
  return a->f[k][(q[0] * g->n[1] + q[1]) * g->n[2] + q[2]];
}

/* ---- local functions: each writes only its own element(s) ---------------- */

/* Fig. 1 generalised with a coefficient c: the figure's right-hand side is
 * U(0,+1) + U(-1,0) - 3 U(0,0) + U(+1,0) + U(0,-1) = u + 1*(N+S+E+W-4u). */
static void lf_jacobi5(const or_acc* a, const double* prm, double* out) {
  double c = prm[0];
  double u = U(a, 0, 0, 0, 0);
  double nb = U(a, 0, -1, 0, 0) + U(a, 0, +1, 0, 0) + U(a, 0, 0, -1, 0) + U(a, 0, 0, +1, 0);
  out[0] = u + c * (nb - 4.0 * u);
}

static void lf_diff7(const or_acc* a, const double* prm, double* out) {
  double c = prm[0];
  double u = U(a, 0, 0, 0, 0);
  double nb = U(a, 0, -1, 0, 0) + U(a, 0, +1, 0, 0) + U(a, 0, 0, -1, 0) + U(a, 0, 0, +1, 0) +
              U(a, 0, 0, 0, -1) + U(a, 0, 0, 0, +1);
  out[0] = u + c * (nb - 6.0 * u);
}

/* Fourth-order 1D Laplacian weights (-1/12, 4/3, -5/2, 4/3, -1/12). */
static double l4x(const or_acc* a) {
  return -1.0 / 12.0 * U(a, 0, -2, 0, 0) + 4.0 / 3.0 * U(a, 0, -1, 0, 0) - 2.5 * U(a, 0, 0, 0, 0) +
         4.0 / 3.0 * U(a, 0, +1, 0, 0) - 1.0 / 12.0 * U(a, 0, +2, 0, 0);
}
static double l4y(const or_acc* a) {
  return -1.0 / 12.0 * U(a, 0, 0, -2, 0) + 4.0 / 3.0 * U(a, 0, 0, -1, 0) - 2.5 * U(a, 0, 0, 0, 0) +
         4.0 / 3.0 * U(a, 0, 0, +1, 0) - 1.0 / 12.0 * U(a, 0, 0, +2, 0);
}

static void lf_star9r2(const or_acc* a, const double* prm, double* out) {
  double c = prm[0];
  out[0] = U(a, 0, 0, 0, 0) + c * (l4x(a) + l4y(a));
}

/* Linearised shallow water on an Arakawa C-grid: h at the cell centre, u on
 * the east face, v on the north face of cell (i,j); forward Euler in time. */
static void lf_swe(const or_acc* a, const double* prm, double* out) {
  double dt = prm[0], gr = prm[1], H = prm[2];
  double div = (U(a, 1, 0, 0, 0) - U(a, 1, -1, 0, 0)) + (U(a, 2, 0, 0, 0) - U(a, 2, 0, -1, 0));
  out[0] = U(a, 0, 0, 0, 0) - dt * H * div;
  out[1] = U(a, 1, 0, 0, 0) - dt * gr * (U(a, 0, +1, 0, 0) - U(a, 0, 0, 0, 0));
  out[2] = U(a, 2, 0, 0, 0) - dt * gr * (U(a, 0, 0, +1, 0) - U(a, 0, 0, 0, 0));
}

/* Nonlinear shallow water on an Arakawa C-grid, forward Euler, unit spacing.
 * Fields: eta = h - H (surface elevation about the mean depth H) at the cell
 * centre, u on the east face and v on the north face of cell (i,j).  This is a
 * non-linear physics operator with products of halo values, the kind of local
 * function the paper's Limitations paragraph (Sec. 5) names.
 *   mass:     eta' = eta - dt [ (F(i) - F(i-1)) + (G(j) - G(j-1)) ],
 *             F = (H + mean of eta across the east face) u,
 *             G = (H + mean of eta across the north face) v;
 *   momentum: u' = u + dt [ f vbar - g d_x eta - u D_x u - vbar D_y u ],
 *             v' = v + dt [ -f ubar - g d_y eta - ubar D_x v - v D_y v ],
 * with d the one-sided difference to the next centre, D the centred
 * difference (half the span), vbar the mean of the four v faces around the u
 * face (reads the corner U(+1,-1)) and ubar the mean of the four u faces
 * around the v face (reads the corner U(-1,+1)). */
static void lf_swe_flux(const or_acc* a, const double* prm, double* out) {
  double dt = prm[0], gr = prm[1], fc = prm[2], H = prm[3];
  double e = U(a, 0, 0, 0, 0), eE = U(a, 0, +1, 0, 0), eW = U(a, 0, -1, 0, 0);
  double eN = U(a, 0, 0, +1, 0), eS = U(a, 0, 0, -1, 0);
  double u = U(a, 1, 0, 0, 0), uW = U(a, 1, -1, 0, 0), uE = U(a, 1, +1, 0, 0);
  double uN = U(a, 1, 0, +1, 0), uS = U(a, 1, 0, -1, 0), uWN = U(a, 1, -1, +1, 0);
  double v = U(a, 2, 0, 0, 0), vS = U(a, 2, 0, -1, 0), vN = U(a, 2, 0, +1, 0);
  double vE = U(a, 2, +1, 0, 0), vW = U(a, 2, -1, 0, 0), vES = U(a, 2, +1, -1, 0);
  double F_e = (H + 0.5 * (e + eE)) * u;
  double F_w = (H + 0.5 * (eW + e)) * uW;
  double G_n = (H + 0.5 * (e + eN)) * v;
  double G_s = (H + 0.5 * (eS + e)) * vS;
  double vbar = 0.25 * ((v + vE) + (vS + vES));
  double ubar = 0.25 * ((u + uW) + (uN + uWN));
  out[0] = e - dt * ((F_e - F_w) + (G_n - G_s));
  out[1] = u + dt * (fc * vbar - gr * (eE - e) - u * 0.5 * (uE - uW) - vbar * 0.5 * (uN - uS));
  out[2] = v + dt * (-fc * ubar - gr * (eN - e) - ubar * 0.5 * (vE - vW) - v * 0.5 * (vN - vS));
}

static void lf_linear(const or_acc* a, int ndim, int r, const double* w, double* out) {
  int zr = ndim == 3 ? r : 0;
  int side = 2 * r + 1;
  double s = 0.0;
  for (int dz = -zr; dz <= zr; dz++)
    for (int dy = -r; dy <= r; dy++)
      for (int dx = -r; dx <= r; dx++) {
        double wt = w[((dz + zr) * side + (dy + r)) * side + (dx + r)];
        if (wt != 0.0) s += wt * U(a, 0, dx, dy, dz);
      }
  out[0] = s;
}

/* d(local function)/dc for the diffusion-form stencils u + c L(u): L(u) with
 * the same halo values as the forward. */
static double lf_dcoef(const or_acc* a, int kind) {
  double u = U(a, 0, 0, 0, 0);
  switch (kind) {
    case OR_JACOBI5:
      return U(a, 0, -1, 0, 0) + U(a, 0, +1, 0, 0) + U(a, 0, 0, -1, 0) + U(a, 0, 0, +1, 0) - 4.0 * u;
    case OR_DIFF7:
      return U(a, 0, -1, 0, 0) + U(a, 0, +1, 0, 0) + U(a, 0, 0, -1, 0) + U(a, 0, 0, +1, 0) +
             U(a, 0, 0, 0, -1) + U(a, 0, 0, 0, +1) - 6.0 * u;
    case OR_STAR9R2:
      return l4x(a) + l4y(a);
    default:
      return 0.0;
  }
}

static int nfields_of(int kind) { return (kind == OR_SWE || kind == OR_SWEFLUX) ? 3 : 1; }
static int stencil_nf(const or_stencil* s) { return s->kind == OR_USER ? s->user_nf : nfields_of(s->kind); }

/* U() in the form a user-written function calls it. */
static double tap(const void* acc, int f, int dx, int dy, int dz) {
  return U((const or_acc*)acc, f, dx, dy, dz);
}

static int make_grid(or_grid* g, int ndim, const int64_t* ext, const int* bc, const double* bval) {
  if (ndim != 2 && ndim != 3) return OR_ERR;
  int off = 3 - ndim;
  for (int ax = 0; ax < 3; ax++) {
    g->n[ax] = 1;
    g->bc[ax][0] = g->bc[ax][1] = OR_PERIODIC;
    g->bval[ax][0] = g->bval[ax][1] = 0.0;
  }
  for (int i = 0; i < ndim; i++) {
    if (ext[i] <= 0) return OR_ERR;
    g->n[off + i] = ext[i];
    g->bc[off + i][0] = bc[2 * i];
    g->bc[off + i][1] = bc[2 * i + 1];
    g->bval[off + i][0] = bval[2 * i];
    g->bval[off + i][1] = bval[2 * i + 1];
  }
  g->ndim = ndim;
  return OR_OK;
}

/* One sweep: out = f(in) at every point, from the frozen snapshot `in`. */
static void sweep(const or_grid* g, const or_stencil* s, double* const* in, double* const* out,
                  int nthreads) {
  int nf = stencil_nf(s);
  int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
  int64_t outer = g->ndim == 3 ? n0 : n1;
  (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int64_t o = 0; o < outer; o++) {
    or_acc a;
    a.g = g;
    for (int k = 0; k < nf; k++) a.f[k] = in[k];
    int64_t z0 = g->ndim == 3 ? o : 0, z1 = g->ndim == 3 ? o + 1 : n0;
    int64_t y0 = g->ndim == 3 ? 0 : o, y1 = g->ndim == 3 ? n1 : o + 1;
    for (int64_t z = z0; z < z1; z++)
      for (int64_t y = y0; y < y1; y++)
        for (int64_t x = 0; x < n2; x++) {
          a.p[0] = z; a.p[1] = y; a.p[2] = x;
          double r[OR_MAXF];
          switch (s->kind) {
            case OR_JACOBI5: lf_jacobi5(&a, s->prm, r); break;
            case OR_DIFF7: lf_diff7(&a, s->prm, r); break;
            case OR_STAR9R2: lf_star9r2(&a, s->prm, r); break;
            case OR_SWE: lf_swe(&a, s->prm, r); break;
            case OR_SWEFLUX: lf_swe_flux(&a, s->prm, r); break;
            case OR_USER: s->user(&a, tap, s->prm, r); break;
            default: lf_linear(&a, g->ndim, s->radius, s->w, r); break;
          }
          int64_t idx = (z * n1 + y) * n2 + x;
          for (int k = 0; k < nf; k++) out[k][idx] = r[k];
        }
  }
}

static int check_stencil(const or_grid* g, const or_stencil* s) {
  switch (s->kind) {
    case OR_JACOBI5: case OR_STAR9R2: case OR_SWE: case OR_SWEFLUX:
      return g->ndim == 2 ? OR_OK : OR_ERR;
    case OR_DIFF7: return g->ndim == 3 ? OR_OK : OR_ERR;
    case OR_LINEAR: return (s->radius >= 0 && s->w) ? OR_OK : OR_ERR;
    case OR_USER: return (s->user && s->user_nf >= 1 && s->user_nf <= OR_MAXF) ? OR_OK : OR_ERR;
    default: return OR_ERR;
  }
}

/* Apply the local function nsteps times.  in/out hold nfields arrays each;
 * `in` is not modified.  nsteps = 0 copies. */
int oracle_apply(int ndim, const int64_t* ext, const int* bc, const double* bval, int kind,
                 const double* prm, int radius, const double* weights, const double* const* in,
                 double* const* out, int64_t nsteps, int nthreads) {
  or_grid g;
  if (make_grid(&g, ndim, ext, bc, bval) != OR_OK) return OR_ERR;
  or_stencil s = {kind, radius, NULL, 0, prm, weights};
  if (check_stencil(&g, &s) != OR_OK) return OR_ERR;
  int nf = nfields_of(kind);
  int64_t n = npoints(&g);
  double* cur[OR_MAXF];
  double* nxt[OR_MAXF];
  for (int k = 0; k < nf; k++) {
    cur[k] = (double*)malloc(sizeof(double) * n);
    nxt[k] = (double*)malloc(sizeof(double) * n);
    if (!cur[k] || !nxt[k]) return OR_ERR;
    memcpy(cur[k], in[k], sizeof(double) * n);
  }
  for (int64_t t = 0; t < nsteps; t++) {
    sweep(&g, &s, cur, nxt, nthreads);
    for (int k = 0; k < nf; k++) { double* tmp = cur[k]; cur[k] = nxt[k]; nxt[k] = tmp; }
  }
  for (int k = 0; k < nf; k++) {
    memcpy(out[k], cur[k], sizeof(double) * n);
    free(cur[k]);
    free(nxt[k]);
  }
  return OR_OK;
}

/* Multi-stage time stepping over the local function.  The local function is
 * itself one forward-Euler step E(u) = u + dt F(u); the strong-stability-
 * preserving Runge-Kutta schemes of Shu and Osher (J. Comput. Phys. 77, 1988)
 * are convex combinations of Euler steps, so every stage is a sweep of the
 * same local function followed by a pointwise combination with the state at
 * the start of the step:
 *   stages = 2:  u1 = E(u);  u+ = 1/2 u + 1/2 E(u1)
 *   stages = 3:  u1 = E(u);  u2 = 3/4 u + 1/4 E(u1);  u+ = 1/3 u + 2/3 E(u2)
 *   stages = 1:  u+ = E(u)   (plain application)
 * The intermediate states u1, u2 are the "intermediate results resulting from
 * multiple intermediate update steps" that the paper's Limitations paragraph
 * (Sec. 5) says LOPe does not store; each stage refreshes the halo from its
 * own input, as the Euler sweep does. */
static void combine(double* dst, double a, const double* base, double b, const double* e,
                    int64_t n) {
  for (int64_t i = 0; i < n; i++) dst[i] = a * base[i] + b * e[i];
}

static int apply_scheme(const or_grid* gp, const or_stencil* sp, int stages,
                        const double* const* in, double* const* out, int64_t nsteps, int nthreads) {
  const or_grid g = *gp;
  const or_stencil s = *sp;
  if (check_stencil(&g, &s) != OR_OK) return OR_ERR;
  if (stages < 1 || stages > 3) return OR_ERR;
  int nf = stencil_nf(&s);
  int64_t n = npoints(&g);
  double *u[OR_MAXF], *st[OR_MAXF], *e[OR_MAXF];
  for (int k = 0; k < nf; k++) {
    u[k] = (double*)malloc(sizeof(double) * n);
    st[k] = (double*)malloc(sizeof(double) * n);
    e[k] = (double*)malloc(sizeof(double) * n);
    if (!u[k] || !st[k] || !e[k]) return OR_ERR;
    memcpy(u[k], in[k], sizeof(double) * n);
  }
  for (int64_t t = 0; t < nsteps; t++) {
    if (stages == 1) {
      sweep(&g, &s, u, e, nthreads);
      for (int k = 0; k < nf; k++) memcpy(u[k], e[k], sizeof(double) * n);
      continue;
    }
    sweep(&g, &s, u, st, nthreads); /* u1 = E(u) */
    sweep(&g, &s, st, e, nthreads); /* E(u1) */
    if (stages == 2) {
      for (int k = 0; k < nf; k++) combine(u[k], 0.5, u[k], 0.5, e[k], n);
    } else {
      for (int k = 0; k < nf; k++) combine(st[k], 0.75, u[k], 0.25, e[k], n); /* u2 */
      sweep(&g, &s, st, e, nthreads);                                         /* E(u2) */
      for (int k = 0; k < nf; k++) combine(u[k], 1.0 / 3.0, u[k], 2.0 / 3.0, e[k], n);
    }
  }
  for (int k = 0; k < nf; k++) {
    memcpy(out[k], u[k], sizeof(double) * n);
    free(u[k]);
    free(st[k]);
    free(e[k]);
  }
  return OR_OK;
}

int oracle_apply_rk(int ndim, const int64_t* ext, const int* bc, const double* bval, int kind,
                    const double* prm, int radius, const double* weights, int stages,
                    const double* const* in, double* const* out, int64_t nsteps, int nthreads) {
  or_grid g;
  if (make_grid(&g, ndim, ext, bc, bval) != OR_OK) return OR_ERR;
  or_stencil s = {kind, radius, NULL, 0, prm, weights};
  return apply_scheme(&g, &s, stages, in, out, nsteps, nthreads);
}

/* A user-written local function `fn` with nf fields (the same text the library
 * compiles for the GPU, compiled here for the host in FP64 by oracle/oracle.py),
 * applied nsteps times with the scheme of `stages` stages. */
int oracle_apply_user(int ndim, const int64_t* ext, const int* bc, const double* bval, int nf,
                      or_user_fn fn, const double* prm, int stages, const double* const* in,
                      double* const* out, int64_t nsteps, int nthreads) {
  or_grid g;
  if (make_grid(&g, ndim, ext, bc, bval) != OR_OK) return OR_ERR;
  or_stencil s = {OR_USER, 0, fn, nf, prm, NULL};
  return apply_scheme(&g, &s, stages, in, out, nsteps, nthreads);
}

/* Weight table of a linear stencil, (2r+1)^ndim entries, slowest offset
 * first, written from each stencil's definition.  Returns the radius, or -1. */
int oracle_weights(int kind, const double* prm, int ndim, int radius, const double* wlin,
                   double* w, int wcap) {
  int r, side, zr;
  switch (kind) {
    case OR_JACOBI5: case OR_DIFF7: r = 1; break;
    case OR_STAR9R2: r = 2; break;
    case OR_LINEAR: r = radius; break;
    default: return -1;
  }
  side = 2 * r + 1;
  zr = ndim == 3 ? r : 0;
  int total = side * side * (2 * zr + 1);
  if (total > wcap) return -1;
  if (kind == OR_LINEAR) {
    memcpy(w, wlin, sizeof(double) * total);
    return r;
  }
  memset(w, 0, sizeof(double) * total);
#define W(dx, dy, dz) w[(((dz) + zr) * side + ((dy) + r)) * side + ((dx) + r)]
  double c = prm[0];
  if (kind == OR_JACOBI5) {
    W(0, 0, 0) = 1.0 - 4.0 * c;
    W(-1, 0, 0) = W(1, 0, 0) = W(0, -1, 0) = W(0, 1, 0) = c;
  } else if (kind == OR_DIFF7) {
    W(0, 0, 0) = 1.0 - 6.0 * c;
    W(-1, 0, 0) = W(1, 0, 0) = W(0, -1, 0) = W(0, 1, 0) = W(0, 0, -1) = W(0, 0, 1) = c;
  } else {
    W(0, 0, 0) = 1.0 + c * (-2.5 - 2.5);
    W(-1, 0, 0) = W(1, 0, 0) = W(0, -1, 0) = W(0, 1, 0) = c * (4.0 / 3.0);
    W(-2, 0, 0) = W(2, 0, 0) = W(0, -2, 0) = W(0, 2, 0) = c * (-1.0 / 12.0);
  }
#undef W
  return r;
}

/* lambda_t = A^T lambda_{t+1}: every point p hands w[o] * lambda_{t+1}[p] to
 * the element its tap o read, i.e. p + o wrapped on periodic axes.  A tap that
 * read a Dirichlet halo value read a constant, so it hands nothing back. */
static void scatter_transpose(const or_grid* g, int r, const double* w, const double* lam_next,
                              double* lam) {
  int64_t n0 = g->n[0], n1 = g->n[1], n2 = g->n[2];
  int zr = g->ndim == 3 ? r : 0;
  int side = 2 * r + 1;
  memset(lam, 0, sizeof(double) * npoints(g));
  for (int64_t z = 0; z < n0; z++)
    for (int64_t y = 0; y < n1; y++)
      for (int64_t x = 0; x < n2; x++) {
        double lp = lam_next[(z * n1 + y) * n2 + x];
        for (int dz = -zr; dz <= zr; dz++)
          for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
              double wt = w[((dz + zr) * side + (dy + r)) * side + (dx + r)];
              if (wt == 0.0) continue;
              int64_t q[3] = {z + dz, y + dy, x + dx};
              int halo_const = 0;
              for (int ax = 0; ax < 3; ax++) {
                if (q[ax] < 0 && g->bc[ax][0] == OR_DIRICHLET) halo_const = 1;
                if (q[ax] >= g->n[ax] && g->bc[ax][1] == OR_DIRICHLET) halo_const = 1;
              }
              if (halo_const) continue;
              for (int ax = 0; ax < 3; ax++) q[ax] = ((q[ax] % g->n[ax]) + g->n[ax]) % g->n[ax];
              lam[(q[0] * n1 + q[1]) * n2 + q[2]] += wt * lp;
            }
      }
}

/* Vector-Jacobian product of u_T = A^T u_0 (T = nsteps): given lambda_T =
 * dL/du_T, returns dL/du_0 and, for the diffusion-form stencils, dL/dc =
 * sum_t <lambda_{t+1}, L u_t>.  Stores the whole trajectory u_0..u_{T-1}. */
int oracle_vjp(int ndim, const int64_t* ext, const int* bc, const double* bval, int kind,
               const double* prm, int radius, const double* weights, const double* u0,
               const double* lamT, int64_t nsteps, double* grad_u0, double* grad_c, int nthreads) {
  or_grid g;
  if (make_grid(&g, ndim, ext, bc, bval) != OR_OK) return OR_ERR;
  or_stencil s = {kind, radius, NULL, 0, prm, weights};
  if (kind == OR_SWE || kind == OR_SWEFLUX || check_stencil(&g, &s) != OR_OK) return OR_ERR;
  int64_t n = npoints(&g);
  double w[125];
  int r = oracle_weights(kind, prm, ndim, radius, weights, w, 125);
  if (r < 0) return OR_ERR;
  double* traj = (double*)malloc(sizeof(double) * n * (size_t)(nsteps + 1));
  double* lam = (double*)malloc(sizeof(double) * n);
  double* lam_prev = (double*)malloc(sizeof(double) * n);
  if (!traj || !lam || !lam_prev) return OR_ERR;
  memcpy(traj, u0, sizeof(double) * n);
  for (int64_t t = 0; t < nsteps; t++) {
    double* in1[1] = {traj + t * n};
    double* out1[1] = {traj + (t + 1) * n};
    sweep(&g, &s, in1, out1, nthreads);
  }
  memcpy(lam, lamT, sizeof(double) * n);
  double gc = 0.0;
  for (int64_t t = nsteps - 1; t >= 0; t--) {
    /* dL/dc += <lambda_{t+1}, L u_t> with L u_t evaluated by the gather. */
    if (kind != OR_LINEAR) {
      or_acc a;
      a.g = &g;
      a.f[0] = traj + t * n;
      for (int64_t z = 0; z < g.n[0]; z++)
        for (int64_t y = 0; y < g.n[1]; y++)
          for (int64_t x = 0; x < g.n[2]; x++) {
            a.p[0] = z; a.p[1] = y; a.p[2] = x;
            gc += lam[(z * g.n[1] + y) * g.n[2] + x] * lf_dcoef(&a, kind);
          }
    }
    scatter_transpose(&g, r, w, lam, lam_prev);
    double* tmp = lam; lam = lam_prev; lam_prev = tmp;
  }
  memcpy(grad_u0, lam, sizeof(double) * n);
  if (grad_c) *grad_c = gc;
  free(traj);
  free(lam);
  free(lam_prev);
  return OR_OK;
}

/* loss = sum (u_T - target)^2 after nsteps; gradients by the discrete adjoint
 * seeded with lambda_T = 2 (u_T - target). */
int oracle_adjoint(int ndim, const int64_t* ext, const int* bc, const double* bval, int kind,
                   const double* prm, int radius, const double* weights, const double* u0,
                   const double* target, int64_t nsteps, double* grad_u0, double* grad_c,
                   double* loss, int nthreads) {
  or_grid g;
  if (make_grid(&g, ndim, ext, bc, bval) != OR_OK) return OR_ERR;
  int64_t n = npoints(&g);
  double* uT = (double*)malloc(sizeof(double) * n);
  double* lamT = (double*)malloc(sizeof(double) * n);
  if (!uT || !lamT) return OR_ERR;
  const double* in1[1] = {u0};
  double* out1[1] = {uT};
  if (oracle_apply(ndim, ext, bc, bval, kind, prm, radius, weights, in1, out1, nsteps, nthreads))
    return OR_ERR;
  double L = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double d = uT[i] - target[i];
    L += d * d;
    lamT[i] = 2.0 * d;
  }
  if (loss) *loss = L;
  int rc = oracle_vjp(ndim, ext, bc, bval, kind, prm, radius, weights, u0, lamT, nsteps, grad_u0,
                      grad_c, nthreads);
  free(uT);
  free(lamT);
  return rc;
}

/* Plain sums used by the invariant checks: sum of a field, and of squares of
 * differences. */
double oracle_sum(const double* x, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += x[i];
  return s;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
