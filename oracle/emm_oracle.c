/*
 * emm_oracle.c -- FP64 CPU oracle of the fictitious-wave-domain, high-order,
 * non-uniform staggered-grid FDTD method of libEMM (Yang, arXiv 2304.00233).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA
 * path is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library: everything below is
 * written independently from the paper's equations.
 *
 * Layout: every 3-D array is [n3][n2][n1] with the x index fastest (Sec. 3.8,
 * "array[k][j][i]").  Padded sizes n_pad = n + 2 (nb + ne) (Sec. 3.4).
 *
 * What it computes, in the paper's order (Algorithm 1 without the airwave
 * step, which is not modelled here):
 *   for it = 0 .. Nt-1:
 *     curl H (with CPML memory, Sec. 3.4 Eq. 22-24)  -> curlH
 *     inject electric source J at t_{n+1/2}           -> curlH - J
 *     update E:  E += dt/eps (curlH - J)              (Sec. 3.1 Eq. 8)
 *     DTFT of E^{n+1} and H^{n+1/2}                   (Sec. 3.5 Eq. 25)
 *     curl E (with CPML memory)                        -> curlE
 *     update H:  H -= dt/mu curlE                     (Eq. 8)
 *   Green's functions (Sec. 2.2 Eq. 7) at receivers and over the volume.
 *
 * Readings of points the paper leaves open are marked "reading:" and listed
 * in the design notes of the repository.
 *
 * Parity pins: every routine here is pinned by CPU tests against closed
 * forms (polynomial exactness and Fornberg's uniform coefficients for the FD
 * weights, the Appendix A dispersion relation for the leapfrog stencil, the
 * analytic whole-space dipole, geometric-series DFT sums, symmetry and
 * reciprocity).
 */
#include <complex.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_MU0 (4.0e-7 * M_PI) /* reading: mu = mu0 everywhere */
#define ORC_MAXK 8              /* 2r knots, r <= 4 */
#define ORC_MAXPT 256           /* sub-dipoles of an antenna */

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EOUTSIDE = 3 };

/* Number of OpenMP threads the loops below use. */
int orc_threads(void)
{
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Vandermonde inversion (Sec. 3.1, Eq. 9-11)                               */
/* ------------------------------------------------------------------------ */

/* Solve V^T(t_0..t_{m-1}) a = f, i.e. find the coefficients a_j of the
 * polynomial p(s) = sum_j a_j s^j with p(t_i) = f_i.  This is the
 * Bjorck-Pereyra route (Golub & Van Loan, Alg. 4.6.1): build the Newton form
 * of the interpolant from divided differences, then expand it into monomials.
 * With t_i = x_i - x, a_0 = f(x) and a_1 = f'(x) (Sec. 3.1). */
static void orc_vander_dual(int m, const double *t, const double *f, double *a)
{
  double col[ORC_MAXK], dd[ORC_MAXK], basis[ORC_MAXK + 1];
  for (int i = 0; i < m; ++i) col[i] = f[i];
  dd[0] = col[0];
  for (int k = 1; k < m; ++k) {           /* divided differences of order k */
    for (int i = 0; i < m - k; ++i)
      col[i] = (col[i + 1] - col[i]) / (t[i + k] - t[i]);
    dd[k] = col[0];                        /* f[t_0, ..., t_k] */
  }
  /* p(s) = sum_k dd[k] * prod_{l<k} (s - t_l); basis holds prod_{l<k}(s - t_l) */
  for (int j = 0; j < m; ++j) a[j] = 0.0;
  for (int j = 0; j <= m; ++j) basis[j] = 0.0;
  basis[0] = 1.0;
  for (int k = 0; k < m; ++k) {
    for (int j = 0; j <= k; ++j) a[j] += dd[k] * basis[j];
    for (int j = k + 1; j >= 1; --j) basis[j] = basis[j - 1] - t[k] * basis[j];
    basis[0] = -t[k] * basis[0];
  }
}

/* Full inverse W = [V^T]^{-1} (row-major, W[row*m + j]) by feeding unit vectors
 * e_j to the solver: the solution is column j of the inverse (Eq. 12). */
void orc_vander_inverse(int m, const double *t, double *W)
{
  double f[ORC_MAXK], a[ORC_MAXK];
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < m; ++i) f[i] = (i == j) ? 1.0 : 0.0;
    orc_vander_dual(m, t, f, a);
    for (int row = 0; row < m; ++row) W[row * m + j] = a[row];
  }
}

/* Weights of row `row` of [V^T(knots - x)]^{-1}: row 0 interpolates f(x),
 * row 1 differentiates f'(x). */
void orc_row_weights(int m, const double *knots, double x, int row, double *w)
{
  double t[ORC_MAXK] = {0}, W[ORC_MAXK * ORC_MAXK];
  for (int i = 0; i < m; ++i) t[i] = knots[i] - x;
  orc_vander_inverse(m, t, W);
  for (int j = 0; j < m; ++j) w[j] = W[row * m + j];
}

/* ------------------------------------------------------------------------ */
/* One grid axis: padding, half nodes, FD tables, CPML slabs                */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n, npad, nbe, rd, nb;
  double *X;    /* npad+1 integer nodes (index npad only defines the last half node) */
  double *Xh;   /* npad half nodes x_{i+1/2} */
  double *cp;   /* D+ rows [npad][2rd]: derivative at Xh[i] from F[i-rd+1 .. i+rd] */
  double *cm;   /* D- rows [npad][2rd]: derivative at X[i] from F[i-rd .. i+rd-1] (half samples) */
  int *slab;    /* [npad] CPML slab index 0..2nb-1 of integer samples X[i], or -1 */
  int *slabh;   /* [npad] CPML slab index 0..2nb-1 of half samples Xh[i], or -1 */
  double *pa_i, *pb_i; /* [2nb] CPML a, b at integer positions */
  double *pa_h, *pb_h; /* [2nb] CPML a, b at half positions */
} orc_axis;

static void orc_axis_free(orc_axis *ax)
{
  free(ax->X); free(ax->Xh); free(ax->cp); free(ax->cm); free(ax->slab); free(ax->slabh);
  free(ax->pa_i); free(ax->pb_i); free(ax->pa_h); free(ax->pb_h);
  memset(ax, 0, sizeof(*ax));
}

/* reading: pads repeat the adjacent edge spacing; the extra node X[npad]
 * defines the last half node (Sec. 3.4 padding, Sec. 5.3 node counts). */
static int orc_axis_nodes(orc_axis *ax, int n, const double *x, int rd, int nb, int ne)
{
  memset(ax, 0, sizeof(*ax));
  if (n < 2) return ORC_EINVAL;
  for (int i = 1; i < n; ++i) if (!(x[i] > x[i - 1])) return ORC_EINVAL;
  ax->n = n; ax->rd = rd; ax->nb = nb; ax->nbe = nb + ne;
  ax->npad = n + 2 * ax->nbe;
  int np = ax->npad, nbe = ax->nbe;
  ax->X = malloc(sizeof(double) * (np + 1));
  ax->Xh = malloc(sizeof(double) * np);
  ax->cp = calloc((size_t)np * 2 * rd, sizeof(double));
  ax->cm = calloc((size_t)np * 2 * rd, sizeof(double));
  ax->slab = malloc(sizeof(int) * np);
  ax->slabh = malloc(sizeof(int) * np);
  ax->pa_i = calloc(2 * nb + 1, sizeof(double)); ax->pb_i = calloc(2 * nb + 1, sizeof(double));
  ax->pa_h = calloc(2 * nb + 1, sizeof(double)); ax->pb_h = calloc(2 * nb + 1, sizeof(double));
  if (!ax->X || !ax->Xh || !ax->cp || !ax->cm || !ax->slab || !ax->slabh) return ORC_ENOMEM;
  double h0 = x[1] - x[0], h1 = x[n - 1] - x[n - 2];
  for (int i = 0; i < n; ++i) ax->X[nbe + i] = x[i];
  for (int m = 1; m <= nbe; ++m) ax->X[nbe - m] = x[0] - m * h0;
  for (int m = 1; m <= nbe + 1; ++m) ax->X[nbe + n - 1 + m] = x[n - 1] + m * h1;
  for (int i = 0; i < np; ++i) ax->Xh[i] = 0.5 * (ax->X[i] + ax->X[i + 1]); /* reading: midpoint */
  /* CPML slabs (Sec. 3.4): nb samples of each kind on each face.  Integer
   * sample i mirrors to np-1-i, half sample i (at Xh[i]) mirrors to np-2-i;
   * reading: the far-side slab of half samples is [np-1-nb, np-2] so that both
   * faces damp the same positions (the last half sample np-1 is never updated). */
  for (int i = 0; i < np; ++i) {
    ax->slab[i] = (i < nb) ? i : (i >= np - nb ? nb + (np - 1 - i) : -1);
    ax->slabh[i] = (i < nb) ? i : ((i >= np - 1 - nb && i <= np - 2) ? nb + (np - 2 - i) : -1);
  }
  return ORC_OK;
}

/* FD tables of Eq. 13-14, reading of which Vandermonde gives which operator:
 *   D+ at Xh[i] uses integer nodes X[i-r+1..i+r] and multiplies F[i-r+1..i+r];
 *   D- at X[i]  uses half nodes Xh[i-r..i+r-1]   and multiplies F[i-r..i+r-1].
 * The grid holds integer samples 0..np-1 and half samples 0..np-2 (reading:
 * the half sample past the last node, index np-1, lies off the grid and is
 * neither updated nor used).  Rows whose knots leave the grid stay zero. */
static void orc_axis_fd(orc_axis *ax)
{
  int r = ax->rd, m = 2 * r, np = ax->npad;
  for (int i = r - 1; i <= np - 1 - r; ++i)
    orc_row_weights(m, &ax->X[i - r + 1], ax->Xh[i], 1, &ax->cp[(size_t)i * m]);
  for (int i = r; i <= np - 1 - r; ++i)
    orc_row_weights(m, &ax->Xh[i - r], ax->X[i], 1, &ax->cm[(size_t)i * m]);
}

/* CPML coefficients (Eq. 23-24) with kappa = 1.  Profile after Komatitsch &
 * Martin (2007): d = d0 (xi/L)^2, d0 = -3 vmax ln(R) / (2L), R = 1e-3,
 * alpha = pi fmax (1 - xi/L); xi is the distance of the sample coordinate
 * into the layer and L the layer thickness on that face. */
static void orc_cpml_ab(const orc_axis *ax, int s, double pos, double vmax, double fmax,
                        double dt, double *a, double *b)
{
  int nb = ax->nb, np = ax->npad;
  double xi, L;
  if (s < nb) { xi = ax->X[nb] - pos; L = ax->X[nb] - ax->X[0]; }
  else        { xi = pos - ax->X[np - 1 - nb]; L = ax->X[np - 1] - ax->X[np - 1 - nb]; }
  if (xi < 0) xi = 0;
  if (xi > L) xi = L;
  double d0 = -3.0 * vmax * log(1e-3) / (2.0 * L);
  double d = d0 * (xi / L) * (xi / L);
  double alpha = M_PI * fmax * (1.0 - xi / L);
  *b = exp(-(d + alpha) * dt);
  *a = (d + alpha > 0) ? d / (d + alpha) * (*b - 1.0) : 0.0;
}

static void orc_axis_cpml(orc_axis *ax, double vmax, double fmax, double dt)
{
  int nb = ax->nb, np = ax->npad;
  for (int s = 0; s < 2 * nb; ++s) {
    int i = (s < nb) ? s : np - 1 - (s - nb);    /* integer sample of slab entry s */
    int ih = (s < nb) ? s : np - 2 - (s - nb);   /* half sample of slab entry s */
    orc_cpml_ab(ax, s, ax->X[i], vmax, fmax, dt, &ax->pa_i[s], &ax->pb_i[s]);
    orc_cpml_ab(ax, s, ax->Xh[ih], vmax, fmax, dt, &ax->pa_h[s], &ax->pb_h[s]);
  }
}

/* D_max of Sec. 3.2 (Eq. 16): the largest absolute row sum of either table. */
static double orc_axis_dmax(const orc_axis *ax)
{
  int r = ax->rd, m = 2 * r, np = ax->npad;
  double dm = 0.0;
  for (int i = r - 1; i <= np - 1 - r; ++i) {
    double s = 0; for (int j = 0; j < m; ++j) s += fabs(ax->cp[(size_t)i * m + j]);
    if (s > dm) dm = s;
  }
  for (int i = r; i <= np - 1 - r; ++i) {
    double s = 0; for (int j = 0; j < m; ++j) s += fabs(ax->cm[(size_t)i * m + j]);
    if (s > dm) dm = s;
  }
  return dm;
}

/* Exported axis tables for the bit-exact index-map and coefficient tests. */
int orc_axis_tables(int n, const double *x, int rd, int nb, int ne,
                    double vmax, double fmax, double dt,
                    double *X, double *Xh, double *cp, double *cm, int *slab, int *slabh,
                    double *pml /* [4][2nb]: a_int, b_int, a_half, b_half */,
                    double *dmax, int *ranges /* [4]: first/last D+ row, first/last D- row */)
{
  orc_axis ax;
  int st = orc_axis_nodes(&ax, n, x, rd, nb, ne);
  if (st) { orc_axis_free(&ax); return st; }
  orc_axis_fd(&ax);
  orc_axis_cpml(&ax, vmax, fmax, dt);
  int np = ax.npad, m = 2 * rd;
  if (X) memcpy(X, ax.X, sizeof(double) * (np + 1));
  if (Xh) memcpy(Xh, ax.Xh, sizeof(double) * np);
  if (cp) memcpy(cp, ax.cp, sizeof(double) * np * m);
  if (cm) memcpy(cm, ax.cm, sizeof(double) * np * m);
  if (slab) memcpy(slab, ax.slab, sizeof(int) * np);
  if (slabh) memcpy(slabh, ax.slabh, sizeof(int) * np);
  if (pml) {
    memcpy(pml + 0 * 2 * nb, ax.pa_i, sizeof(double) * 2 * nb);
    memcpy(pml + 1 * 2 * nb, ax.pb_i, sizeof(double) * 2 * nb);
    memcpy(pml + 2 * 2 * nb, ax.pa_h, sizeof(double) * 2 * nb);
    memcpy(pml + 3 * 2 * nb, ax.pb_h, sizeof(double) * 2 * nb);
  }
  if (dmax) *dmax = orc_axis_dmax(&ax);
  if (ranges) { ranges[0] = rd - 1; ranges[1] = np - 1 - rd; ranges[2] = rd; ranges[3] = np - 1 - rd; }
  orc_axis_free(&ax);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Staggering, sources and receivers                                         */
/* ------------------------------------------------------------------------ */

/* Yee staggering: component c in {Ex,Ey,Ez,Hx,Hy,Hz} sits on half nodes along
 * these axes (1) and on integer nodes along the others (0). */
static const int ORC_HALF[6][3] = {
  {1, 0, 0}, {0, 1, 0}, {0, 0, 1},   /* Ex, Ey, Ez */
  {0, 1, 1}, {1, 0, 1}, {1, 1, 0},   /* Hx, Hy, Hz */
};

/* reading (Sec. 3.1 and 5.3, arbitrary source/receiver positions): along each
 * axis take the component's own node array P (X or Xh), i = max{i: P[i] <= p},
 * knots i-r+1 .. i+r; all knots must lie outside the CPML slabs.  Weights are
 * row 0 of [V^T]^{-1} (Lagrange interpolation), tensor product over axes. */
static int orc_locate_axis(const orc_axis *ax, int half, double p, int *start, double *w)
{
  const double *P = half ? ax->Xh : ax->X;
  int r = ax->rd, np = ax->npad, nb = ax->nb;
  if (!(p >= P[0])) return ORC_EOUTSIDE;
  int i = 0;
  for (int k = 0; k < np; ++k) if (P[k] <= p) i = k;
  int s = i - r + 1;
  if (s < nb || i + r > np - 1 - nb) return ORC_EOUTSIDE;
  *start = s;
  orc_row_weights(2 * r, &P[s], p, 0, w);
  return ORC_OK;
}

typedef struct { int start[3]; double w[3][ORC_MAXK]; } orc_stencil;

/* Exported for the index-map tests: stencil start per axis and 1-D weights. */
int orc_locate(int n1, const double *x1, int n2, const double *x2, int n3, const double *x3,
               int rd, int nb, int ne, int comp, const double *pos, int *start, double *w)
{
  orc_axis ax[3];
  const int n[3] = {n1, n2, n3};
  const double *xs[3] = {x1, x2, x3};
  int st = ORC_OK;
  memset(ax, 0, sizeof(ax));
  for (int a = 0; a < 3 && !st; ++a) st = orc_axis_nodes(&ax[a], n[a], xs[a], rd, nb, ne);
  for (int a = 0; a < 3 && !st; ++a)
    st = orc_locate_axis(&ax[a], ORC_HALF[comp][a], pos[a], &start[a], &w[a * 2 * rd]);
  for (int a = 0; a < 3; ++a) orc_axis_free(&ax[a]);
  return st;
}

/* ------------------------------------------------------------------------ */
/* The forward problem                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n[3];
  const double *x[3];        /* interior node coordinates per axis */
  int rd, nb, ne;
  const double *sigma;       /* [3][n3][n2][n1] staggered sigma_xx, sigma_yy, sigma_zz */
  double omega0;             /* fictitious transform: eps = sigma / (2 omega0) */
  double sigma_min;          /* <= 0: min of sigma (sets vmax for CFL and CPML) */
  double dt;                 /* <= 0: 0.99 / eta */
  int nt;
  double fmax;               /* wavelet bandwidth and CPML alpha */
  double src[3];
  double az, dip, moment;
  int nrec;
  const double *rec;         /* [nrec][3] */
  int nfreq;
  const double *freqs;       /* Hz */
  int want_volume;
  int convergence;           /* 1: stop early by the corner test (every 100 steps) */
  int inject;                /* 0: no source term */
  int pml;                   /* 0: no CPML memory terms */
  const double *init_fields; /* [6][n3p][n2p][n1p] E then H (H at t_{1/2}), or NULL */
  double *final_fields;      /* same layout, or NULL */
  /* outputs (caller-owned, may be NULL) */
  double *rec_G;             /* [nrec][6][nfreq][2] Green's functions */
  double *rec_acc;           /* [nrec][6][nfreq][2] raw DTFT accumulators */
  double *jhat;              /* [nfreq][2] source spectrum */
  double *vol_G;             /* [6][nfreq][n3][n2][n1][2] Green's functions on the interior */
  double *info;              /* [4]: dt, vmax, nt actually run, eta */
  /* optional sampled volume DTFT: flat indices into [6][n3][n2][n1] */
  int nvs;
  const long long *vs_idx;
  double *vs_G;              /* [nvs][nfreq][2] Green's functions at those samples */
  int magnetic;              /* 1: the source is a magnetic dipole M, injected in
                                the H update (Eq. 5); 0: an electric dipole J */
  double src_length;         /* > 0: an antenna of this length (m) along the
                                dipole direction, centred at src */
  int src_points;            /* its sub-dipoles (used when src_length > 0) */
  int airwave;               /* 1: the top interior node is an interface with
                                air (Sec. 3.3), no CPML on the top face */
} orc_problem;

typedef struct {
  orc_axis ax[3];
  int np[3], rd;
  size_t ncell;
  double *F[6];       /* Ex Ey Ez Hx Hy Hz */
  double *C[3];       /* curl work arrays */
  double *ie[3];      /* dt / eps_ii = 2 omega0 dt / sigma_ii on the padded grid */
  double *psi[12];    /* CPML memory, full-size (only slab entries are used) */
} orc_state;

#define IDX(st, k, j, i) (((size_t)(k) * (st)->np[1] + (size_t)(j)) * (st)->np[0] + (size_t)(i))

static int orc_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Valid range of the sample index along axis a for a component whose
 * derivative needs D- (E update) or D+ (H update) along that axis (reading:
 * a sample is updated only if every stencil it uses lies on the grid, i.e.
 * integer samples 0..np-1 and half samples 0..np-2). */
static void orc_range_Dm(const orc_state *st, int a, int *lo, int *hi)
{ *lo = st->rd; *hi = st->np[a] - 1 - st->rd; }
static void orc_range_Dp(const orc_state *st, int a, int *lo, int *hi)
{ *lo = st->rd - 1; *hi = st->np[a] - 1 - st->rd; }

/* D- along axis a of field G at sample (i,j,k) (half samples -> integer position). */
static double orc_dm(const orc_state *st, int a, const double *G, int i, int j, int k)
{
  int r = st->rd, m = 2 * r;
  int c = (a == 0) ? i : (a == 1 ? j : k);
  const double *w = &st->ax[a].cm[(size_t)c * m];
  double s = 0.0;
  for (int q = 0; q < m; ++q) {
    int ii = i, jj = j, kk = k;
    if (a == 0) ii = i - r + q; else if (a == 1) jj = j - r + q; else kk = k - r + q;
    s += w[q] * G[IDX(st, kk, jj, ii)];
  }
  return s;
}

/* D+ along axis a (integer samples -> half position). */
static double orc_dp(const orc_state *st, int a, const double *G, int i, int j, int k)
{
  int r = st->rd, m = 2 * r;
  int c = (a == 0) ? i : (a == 1 ? j : k);
  const double *w = &st->ax[a].cp[(size_t)c * m];
  double s = 0.0;
  for (int q = 0; q < m; ++q) {
    int ii = i, jj = j, kk = k;
    if (a == 0) ii = i - r + 1 + q; else if (a == 1) jj = j - r + 1 + q; else kk = k - r + 1 + q;
    s += w[q] * G[IDX(st, kk, jj, ii)];
  }
  return s;
}

/* CPML memory update psi <- b psi + a d, returns d + psi (Eq. 22-23). */
static double orc_pml(const orc_state *st, int pml, int a, int half, int c, double *psi,
                      size_t idx, double d)
{
  if (!pml) return d;
  int s = half ? st->ax[a].slabh[c] : st->ax[a].slab[c];
  if (s < 0) return d;
  double aa = half ? st->ax[a].pa_h[s] : st->ax[a].pa_i[s];
  double bb = half ? st->ax[a].pb_h[s] : st->ax[a].pb_i[s];
  psi[idx] = bb * psi[idx] + aa * d;
  return d + psi[idx];
}

/* curl H at E positions (Sec. 3.4, curl assembly):
 *   (curl H)_x = D-_y Hz - D-_z Hy, (curl H)_y = D-_z Hx - D-_x Hz,
 *   (curl H)_z = D-_x Hy - D-_y Hx. */
static void orc_curl_H(orc_state *st, int pml)
{
  const double *Hx = st->F[3], *Hy = st->F[4], *Hz = st->F[5];
  for (int c = 0; c < 3; ++c) {
    /* derivative axes p (positive term) and q (negative term) of component c */
    int p = (c + 1) % 3, q = (c + 2) % 3;
    const double *Gp = st->F[3 + q];   /* (curl H)_c = D_p H_q - D_q H_p */
    const double *Gq = st->F[3 + p];
    int lo[3], hi[3];
    lo[c] = 0; hi[c] = st->np[c] - 2;   /* E_c: half samples along its own axis */
    orc_range_Dm(st, p, &lo[p], &hi[p]);
    orc_range_Dm(st, q, &lo[q], &hi[q]);
    double *C = st->C[c];
    double *psip = st->psi[2 * c], *psiq = st->psi[2 * c + 1];
    memset(C, 0, sizeof(double) * st->ncell);
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t id = IDX(st, k, j, i);
          int cc[3] = {i, j, k};
          double dp = orc_dm(st, p, Gp, i, j, k);
          double dq = orc_dm(st, q, Gq, i, j, k);
          dp = orc_pml(st, pml, p, 0, cc[p], psip, id, dp);
          dq = orc_pml(st, pml, q, 0, cc[q], psiq, id, dq);
          C[id] = dp - dq;
        }
  }
  (void)Hx; (void)Hy; (void)Hz;
}

/* curl E at H positions:
 *   (curl E)_x = D+_y Ez - D+_z Ey, (curl E)_y = D+_z Ex - D+_x Ez,
 *   (curl E)_z = D+_x Ey - D+_y Ex. */
static void orc_curl_E(orc_state *st, int pml)
{
  for (int c = 0; c < 3; ++c) {
    int p = (c + 1) % 3, q = (c + 2) % 3;
    const double *Gp = st->F[q];       /* (curl E)_c = D_p E_q - D_q E_p */
    const double *Gq = st->F[p];
    int lo[3], hi[3];
    lo[c] = 0; hi[c] = st->np[c] - 1;
    orc_range_Dp(st, p, &lo[p], &hi[p]);
    orc_range_Dp(st, q, &lo[q], &hi[q]);
    double *C = st->C[c];
    double *psip = st->psi[6 + 2 * c], *psiq = st->psi[6 + 2 * c + 1];
    memset(C, 0, sizeof(double) * st->ncell);
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t id = IDX(st, k, j, i);
          int cc[3] = {i, j, k};
          double dp = orc_dp(st, p, Gp, i, j, k);
          double dq = orc_dp(st, q, Gq, i, j, k);
          dp = orc_pml(st, pml, p, 1, cc[p], psip, id, dp);
          dq = orc_pml(st, pml, q, 1, cc[q], psiq, id, dq);
          C[id] = dp - dq;
        }
  }
}

/* E^{n+1} = E^n + dt/eps (curl H - J), on the samples the D- stencils allow. */
static void orc_update_E(orc_state *st)
{
  for (int c = 0; c < 3; ++c) {
    int p = (c + 1) % 3, q = (c + 2) % 3, lo[3], hi[3];
    lo[c] = 0; hi[c] = st->np[c] - 2;
    orc_range_Dm(st, p, &lo[p], &hi[p]);
    orc_range_Dm(st, q, &lo[q], &hi[q]);
    double *E = st->F[c];
    const double *C = st->C[c], *ie = st->ie[c];
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t id = IDX(st, k, j, i);
          E[id] += ie[id] * C[id];
        }
  }
}

/* H^{n+3/2} = H^{n+1/2} - dt/mu0 curl E^{n+1}. */
static void orc_update_H(orc_state *st, double dt)
{
  double f = dt / ORC_MU0;
  for (int c = 0; c < 3; ++c) {
    int p = (c + 1) % 3, q = (c + 2) % 3, lo[3], hi[3];
    lo[c] = 0; hi[c] = st->np[c] - 1;
    orc_range_Dp(st, p, &lo[p], &hi[p]);
    orc_range_Dp(st, q, &lo[q], &hi[q]);
    double *H = st->F[3 + c];
    const double *C = st->C[c];
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t id = IDX(st, k, j, i);
          H[id] -= f * C[id];
        }
  }
}

static double orc_sample(const orc_state *st, const double *F, const orc_stencil *s)
{
  int m = 2 * st->rd;
  double v = 0.0;
  for (int c = 0; c < m; ++c)
    for (int b = 0; b < m; ++b)
      for (int a = 0; a < m; ++a)
        v += s->w[2][c] * s->w[1][b] * s->w[0][a] *
             F[IDX(st, s->start[2] + c, s->start[1] + b, s->start[0] + a)];
  return v;
}

/* Source wavelet, reading: Gaussian exp(-(pi fmax (t - t0))^2), t0 = 1.5/fmax. */
/* Factor of component c (0..5) in the Green's functions.  Eq. 7 for an
 * electric source: G^EE = sE E'/J', G^HE = H'/J', sE = sqrt(-i w/(2 w0)).
 * Reading, for a magnetic source, from the correspondence of Eq. 5 (E' = E,
 * H' = sE H, M' = M): G^EH = E'/M', G^HH = H'/(sE M'). */
static double complex orc_norm(int c, double complex sE, int magnetic)
{
  if (!magnetic) return c < 3 ? sE : 1.0;
  return c < 3 ? 1.0 : 1.0 / sE;
}

static double orc_wavelet(double t, double fmax)
{
  double u = M_PI * fmax * (t - 1.5 / fmax);
  return exp(-u * u);
}

static void orc_state_free(orc_state *st)
{
  for (int a = 0; a < 3; ++a) orc_axis_free(&st->ax[a]);
  for (int c = 0; c < 6; ++c) free(st->F[c]);
  for (int c = 0; c < 3; ++c) { free(st->C[c]); free(st->ie[c]); }
  for (int c = 0; c < 12; ++c) free(st->psi[c]);
}

/* ------------------------------------------------------------------------ */
/* Top boundary with air (Sec. 3.3)                                          */
/* ------------------------------------------------------------------------ */
/* Reading.  The top interior z node k_s = nb + ne is the interface; above it
 * the air has sigma = 0 and no source, so curl H = 0 and div H = 0 (H =
 * -grad phi, phi harmonic) and every component of E is harmonic (Delta E =
 * 0).  A harmonic field that vanishes far above the interface is, for each
 * horizontal wavenumber k = (kx, ky), f(k, z) = f(k, z_s) e^{-|k| h} at the
 * height h = z_s - z above it (z down).  With phi = -H_z / |k| at z_s:
 *   H_x(k) = i kx / |k| H_z(k),   H_y(k) = i ky / |k| H_z(k)
 * (the relations of Sec. 3.3), times e^{-i kx dx / 2} (e^{-i ky dy / 2}) to
 * move from H_z's half x (y) position to H_x's (H_y's) integer one; the
 * k = 0 term of H_x, H_y is 0.  The transform is the 2-D DFT of the whole
 * padded x-y plane (uniform spacing dx, dy, as the FFT of the paper needs),
 * kx = 2 pi p / (nx dx) with p taken in (-nx/2, nx/2]; the extrapolated
 * values are the real part of the inverse. */
static double orc_wavenumber(int p, int n, double d)
{
  return 2.0 * M_PI * (p <= n / 2 ? p : p - n) / (n * d);
}

/* out[q][p] = sum_{j,i} in[j][i] e^{sgn 2 pi i (p i / nx + q j / ny)}, with
 * the twiddles e^{sgn 2 pi i m / n} tabulated for m = 0 .. n-1 */
static void orc_dft2(int nx, int ny, const double complex *in, double complex *out, int sgn)
{
  double complex *t = malloc(sizeof(double complex) * (size_t)nx * ny);
  double complex *wx = malloc(sizeof(double complex) * nx), *wy = malloc(sizeof(double complex) * ny);
  for (int m = 0; m < nx; ++m) wx[m] = cexp(sgn * 2.0 * M_PI * I * m / nx);
  for (int m = 0; m < ny; ++m) wy[m] = cexp(sgn * 2.0 * M_PI * I * m / ny);
  for (int j = 0; j < ny; ++j)
    for (int p = 0; p < nx; ++p) {
      double complex s = 0;
      for (int i = 0; i < nx; ++i) s += in[(size_t)j * nx + i] * wx[(long)p * i % nx];
      t[(size_t)j * nx + p] = s;
    }
  for (int q = 0; q < ny; ++q)
    for (int p = 0; p < nx; ++p) {
      double complex s = 0;
      for (int j = 0; j < ny; ++j) s += t[(size_t)j * nx + p] * wy[(long)q * j % ny];
      out[(size_t)q * nx + p] = s;
    }
  free(t); free(wx); free(wy);
}

/* The air extrapolation of one interface plane in [ny][nx].  kind 0: out[r]
 * = the same E component at the height h[r]; kind 1 (in = H_z): out[2r] =
 * H_x and out[2r+1] = H_y at the height h[r], at their own x-y positions.
 * out holds nh (kind 0) or 2 nh (kind 1) planes [ny][nx]. */
int orc_air_extrapolate(int nx, int ny, double dx, double dy, const double *in, int nh, const double *h,
                        int kind, double *out)
{
  if (nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0) || nh < 0 || (kind != 0 && kind != 1)) return ORC_EINVAL;
  size_t n = (size_t)nx * ny;
  double complex *a = malloc(sizeof(double complex) * n), *F = malloc(sizeof(double complex) * n);
  double complex *G = malloc(sizeof(double complex) * n), *g = malloc(sizeof(double complex) * n);
  for (size_t q = 0; q < n; ++q) a[q] = in[q];
  orc_dft2(nx, ny, a, F, -1);
  for (int r = 0; r < nh; ++r)
    for (int o = 0; o < (kind ? 2 : 1); ++o) {
      for (int q = 0; q < ny; ++q)
        for (int p = 0; p < nx; ++p) {
          double kx = orc_wavenumber(p, nx, dx), ky = orc_wavenumber(q, ny, dy), kk = sqrt(kx * kx + ky * ky);
          double complex f = exp(-kk * h[r]);
          if (kind == 1)
            f *= kk > 0 ? (o == 0 ? I * kx / kk * cexp(-I * kx * dx / 2) : I * ky / kk * cexp(-I * ky * dy / 2)) : 0.0;
          G[(size_t)q * nx + p] = F[(size_t)q * nx + p] * f;
        }
      orc_dft2(nx, ny, G, g, +1);
      double *dst = out + (size_t)(kind ? 2 * r + o : r) * n;
      for (size_t q = 0; q < n; ++q) dst[q] = creal(g[q]) / (double)n;
    }
  free(a); free(F); free(G); free(g);
  return ORC_OK;
}

/* After the E update: E_x, E_y on the rd - 1 integer rows above the interface. */
static void orc_airwave_E(orc_state *st)
{
  const orc_axis *az = &st->ax[2];
  int nx = st->np[0], ny = st->np[1], ks = az->nbe, nh = st->rd - 1;
  if (nh < 1) return;
  double h[ORC_MAXK], dx = st->ax[0].X[1] - st->ax[0].X[0], dy = st->ax[1].X[1] - st->ax[1].X[0];
  for (int r = 0; r < nh; ++r) h[r] = az->X[ks] - az->X[ks - 1 - r];
  size_t n = (size_t)nx * ny;
  double *in = malloc(sizeof(double) * n), *out = malloc(sizeof(double) * n * nh);
  for (int c = 0; c < 2; ++c) {
    memcpy(in, st->F[c] + IDX(st, ks, 0, 0), sizeof(double) * n);
    orc_air_extrapolate(nx, ny, dx, dy, in, nh, h, 0, out);
    for (int r = 0; r < nh; ++r) memcpy(st->F[c] + IDX(st, ks - 1 - r, 0, 0), out + (size_t)r * n, sizeof(double) * n);
  }
  free(in); free(out);
}

/* After the H update: H_x, H_y on the rd half rows above the interface (half
 * row k sits at Xh[k] = z_{k+1/2}), from H_z on the interface row. */
static void orc_airwave_H(orc_state *st)
{
  const orc_axis *az = &st->ax[2];
  int nx = st->np[0], ny = st->np[1], ks = az->nbe, nh = st->rd;
  double h[ORC_MAXK], dx = st->ax[0].X[1] - st->ax[0].X[0], dy = st->ax[1].X[1] - st->ax[1].X[0];
  for (int r = 0; r < nh; ++r) h[r] = az->X[ks] - az->Xh[ks - 1 - r];
  size_t n = (size_t)nx * ny;
  double *in = malloc(sizeof(double) * n), *out = malloc(sizeof(double) * n * 2 * nh);
  memcpy(in, st->F[5] + IDX(st, ks, 0, 0), sizeof(double) * n);
  orc_air_extrapolate(nx, ny, dx, dy, in, nh, h, 1, out);
  for (int r = 0; r < nh; ++r) {
    memcpy(st->F[3] + IDX(st, ks - 1 - r, 0, 0), out + (size_t)(2 * r) * n, sizeof(double) * n);
    memcpy(st->F[4] + IDX(st, ks - 1 - r, 0, 0), out + (size_t)(2 * r + 1) * n, sizeof(double) * n);
  }
  free(in); free(out);
}

/* Is the padded axis uniformly spaced (relative tolerance 1e-9)? */
static int orc_axis_uniform(const orc_axis *ax)
{
  double d = ax->X[1] - ax->X[0];
  for (int i = 1; i <= ax->npad; ++i)
    if (fabs((ax->X[i] - ax->X[i - 1]) - d) > 1e-9 * d) return 0;
  return 1;
}

int orc_forward(orc_problem *P)
{
  orc_state S, *st = &S;
  memset(st, 0, sizeof(S));
  int rd = P->rd, nb = P->nb, ne = P->ne, st_code = ORC_OK;
  if (rd < 1 || rd > 4 || nb < rd || ne < 0 || P->nt < 0 || P->omega0 <= 0) return ORC_EINVAL;
  st->rd = rd;
  for (int a = 0; a < 3; ++a) {
    st_code = orc_axis_nodes(&st->ax[a], P->n[a], P->x[a], rd, nb, ne);
    if (st_code) { orc_state_free(st); return st_code; }
    orc_axis_fd(&st->ax[a]);
    st->np[a] = st->ax[a].npad;
  }
  st->ncell = (size_t)st->np[0] * st->np[1] * st->np[2];
  size_t nint = (size_t)P->n[0] * P->n[1] * P->n[2];

  /* vmax = 1/sqrt(mu eps), eps = sigma/(2 omega0)  (Sec. 2.2 and Eq. 15) */
  double smin = P->sigma_min;
  if (smin <= 0) {
    smin = INFINITY;
    for (size_t q = 0; q < 3 * nint; ++q) if (P->sigma[q] < smin) smin = P->sigma[q];
  }
  for (size_t q = 0; q < 3 * nint; ++q)
    if (!(P->sigma[q] > 0) || !isfinite(P->sigma[q])) { orc_state_free(st); return ORC_EINVAL; }
  double vmax = sqrt(2.0 * P->omega0 / (ORC_MU0 * smin));
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) { double dm = orc_axis_dmax(&st->ax[a]); d2 += dm * dm; }
  double eta = 0.5 * vmax * sqrt(d2);
  double dt = (P->dt > 0) ? P->dt : 0.99 / eta;   /* Sec. 3.2: dt = 0.99 / eta */
  for (int a = 0; a < 3; ++a) orc_axis_cpml(&st->ax[a], vmax, P->fmax, dt);
  if (P->airwave) {
    /* the FFT of Sec. 3.3 needs uniform x and y; no CPML on the top face */
    if (!orc_axis_uniform(&st->ax[0]) || !orc_axis_uniform(&st->ax[1])) { orc_state_free(st); return ORC_EINVAL; }
    for (int s = 0; s < nb; ++s) {
      st->ax[2].pa_i[s] = st->ax[2].pb_i[s] = 0.0;
      st->ax[2].pa_h[s] = st->ax[2].pb_h[s] = 0.0;
    }
  }

  for (int c = 0; c < 6; ++c) st->F[c] = calloc(st->ncell, sizeof(double));
  for (int c = 0; c < 3; ++c) {
    st->C[c] = calloc(st->ncell, sizeof(double));
    st->ie[c] = calloc(st->ncell, sizeof(double));
  }
  for (int c = 0; c < 12; ++c) st->psi[c] = P->pml ? calloc(st->ncell, sizeof(double)) : NULL;
  for (int c = 0; c < 6; ++c) if (!st->F[c]) { orc_state_free(st); return ORC_ENOMEM; }

  /* Model extension into the pads by edge replication (Sec. 3.8, extend_model),
   * then dt/eps = 2 omega0 dt / sigma. */
  int nbe = nb + ne;
  for (int c = 0; c < 3; ++c) {
    const double *sg = P->sigma + c * nint;
    for (int k = 0; k < st->np[2]; ++k)
      for (int j = 0; j < st->np[1]; ++j)
        for (int i = 0; i < st->np[0]; ++i) {
          int kk = orc_clampi(k - nbe, 0, P->n[2] - 1);
          int jj = orc_clampi(j - nbe, 0, P->n[1] - 1);
          int ii = orc_clampi(i - nbe, 0, P->n[0] - 1);
          double s = sg[((size_t)kk * P->n[1] + jj) * P->n[0] + ii];
          st->ie[c][IDX(st, k, j, i)] = 2.0 * P->omega0 * dt / s;
        }
  }
  if (P->init_fields)
    for (int c = 0; c < 6; ++c) memcpy(st->F[c], P->init_fields + c * st->ncell, sizeof(double) * st->ncell);

  /* Source stencils (only components with a nonzero direction cosine): on
   * the E samples of an electric dipole, on the H samples of a magnetic one
   * (sc = 3).  Reading of the antenna of finite length (Sec. 7: the current
   * spread uniformly over its length): src_points sub-dipoles at the
   * midpoints of equal segments along the dipole direction, each carrying
   * 1/src_points of the moment. */
  double dir[3] = {cos(P->dip) * cos(P->az), cos(P->dip) * sin(P->az), sin(P->dip)};
  int npt = P->src_length > 0 ? P->src_points : 1;
  if (npt < 1 || npt > ORC_MAXPT) { orc_state_free(st); return ORC_EINVAL; }
  orc_stencil *sst = calloc((size_t)npt * 3, sizeof(orc_stencil));
  double *jw[ORC_MAXPT * 3];            /* [point][c]: dir_c * w / (V npt) per stencil node */
  for (int q = 0; q < npt * 3; ++q) jw[q] = NULL;
  int m = 2 * rd, sc = P->magnetic ? 3 : 0;
  if (P->inject) {
    for (int k = 0; k < npt; ++k) {
      double pos[3];
      const double off = P->src_length > 0 ? (-0.5 + (k + 0.5) / npt) * P->src_length : 0.0;
      for (int a = 0; a < 3; ++a) pos[a] = P->src[a] + off * dir[a];
      for (int c = 0; c < 3; ++c) {
        if (dir[c] == 0.0) continue;
        orc_stencil *ss = &sst[k * 3 + c];
        for (int a = 0; a < 3; ++a) {
          st_code = orc_locate_axis(&st->ax[a], ORC_HALF[c + sc][a], pos[a], &ss->start[a], ss->w[a]);
          /* with air above the model, the source stencil stays below the interface */
          if (!st_code && P->airwave && a == 2 && ss->start[2] < st->ax[2].nbe) st_code = ORC_EOUTSIDE;
          if (st_code) {
            for (int q = 0; q < npt * 3; ++q) free(jw[q]);
            free(sst);
            orc_state_free(st);
            return st_code;
          }
        }
        double *wk = jw[k * 3 + c] = malloc(sizeof(double) * m * m * m);
        /* reading: J_node = p s(t) w_node / V_node with V the dual-cell volume
         * of the staggered sample: along a half-node axis X[i+1]-X[i], along
         * an integer-node axis Xh[i]-Xh[i-1]. */
        for (int q3 = 0; q3 < m; ++q3)
          for (int q2 = 0; q2 < m; ++q2)
            for (int q1 = 0; q1 < m; ++q1) {
              int id3[3] = {ss->start[0] + q1, ss->start[1] + q2, ss->start[2] + q3};
              double V = 1.0;
              for (int a = 0; a < 3; ++a) {
                const orc_axis *ax = &st->ax[a];
                V *= ORC_HALF[c + sc][a] ? (ax->X[id3[a] + 1] - ax->X[id3[a]])
                                         : (ax->Xh[id3[a]] - ax->Xh[id3[a] - 1]);
              }
              wk[(q3 * m + q2) * m + q1] = dir[c] * ss->w[0][q1] * ss->w[1][q2] * ss->w[2][q3] / V / npt;
            }
      }
    }
  }

  /* Receiver stencils for the six components. */
  int nrec = P->nrec, nf = P->nfreq;
  orc_stencil *rst = calloc((size_t)(nrec > 0 ? nrec : 1) * 6, sizeof(orc_stencil));
  for (int r = 0; r < nrec; ++r)
    for (int c = 0; c < 6; ++c)
      for (int a = 0; a < 3; ++a) {
        st_code = orc_locate_axis(&st->ax[a], ORC_HALF[c][a], P->rec[3 * r + a],
                                  &rst[r * 6 + c].start[a], rst[r * 6 + c].w[a]);
        if (st_code) {
          free(rst);
          for (int q = 0; q < npt * 3; ++q) free(jw[q]);
          free(sst);
          orc_state_free(st);
          return st_code;
        }
      }

  /* DTFT (Sec. 3.5, Eq. 25) with omega' = (1+i) sqrt(omega omega0) (Eq. 4) and,
   * reading, the dt factor of the integral in Eq. 6 and these time labels:
   * E^{n+1} at (n+1) dt, H^{n+1/2} and J at (n+1/2) dt. */
  double complex *wp = malloc(sizeof(double complex) * (nf > 0 ? nf : 1));
  for (int f = 0; f < nf; ++f) wp[f] = (1.0 + I) * sqrt(2.0 * M_PI * P->freqs[f] * P->omega0);
  double complex *acc = calloc((size_t)(nrec > 0 ? nrec : 1) * 6 * (nf > 0 ? nf : 1), sizeof(double complex));
  double complex *jh = calloc(nf > 0 ? nf : 1, sizeof(double complex));
  double *rval = calloc((size_t)(nrec > 0 ? nrec : 1) * 6, sizeof(double));
  double complex *vol = NULL;
  double complex *vsa = NULL;
  if (P->nvs > 0) vsa = calloc((size_t)P->nvs * nf, sizeof(double complex));
  if (P->want_volume) {
    vol = calloc(6 * (size_t)nf * nint, sizeof(double complex));
    if (!vol) {
      free(rst); free(wp); free(acc); free(jh); free(rval);
      for (int q = 0; q < npt * 3; ++q) free(jw[q]);
      free(sst);
      orc_state_free(st);
      return ORC_ENOMEM;
    }
  }
  /* 8 corners of the interior cube, lowest frequency, all 6 components (A18). */
  int flo = 0;
  for (int f = 1; f < nf; ++f) if (P->freqs[f] < P->freqs[flo]) flo = f;
  double complex corner[8][6], corner_prev[8][6];
  memset(corner, 0, sizeof(corner));

  int nt_run = P->nt;
  for (int it = 0; it < P->nt; ++it) {
    double tJ = (it + 0.5) * dt, tE = (it + 1.0) * dt, tH = (it + 0.5) * dt;
    orc_curl_H(st, P->pml);
    /* reading: J is sampled at t_{n+1/2} (the E update's centre), M at
     * t_{n+1} (the H update's centre) */
    double amp = P->moment * orc_wavelet(P->magnetic ? tE : tJ, P->fmax);
    if (P->inject && !P->magnetic) {
      for (int q = 0; q < npt * 3; ++q) {
        if (!jw[q]) continue;
        const int c = q % 3;
        for (int q3 = 0; q3 < m; ++q3)
          for (int q2 = 0; q2 < m; ++q2)
            for (int q1 = 0; q1 < m; ++q1)
              st->C[c][IDX(st, sst[q].start[2] + q3, sst[q].start[1] + q2, sst[q].start[0] + q1)]
                  -= amp * jw[q][(q3 * m + q2) * m + q1];
      }
    }
    orc_update_E(st);
    if (P->airwave) orc_airwave_E(st);
    /* receiver values: E^{n+1} (just updated) and H^{n+1/2} (not yet updated) */
    for (int r = 0; r < nrec; ++r)
      for (int c = 0; c < 6; ++c) rval[r * 6 + c] = orc_sample(st, st->F[c], &rst[r * 6 + c]);
    for (int f = 0; f < nf; ++f) {
      double complex fE = cexp(I * wp[f] * tE) * dt;
      double complex fH = cexp(I * wp[f] * tH) * dt;
      jh[f] += cexp(I * wp[f] * (P->magnetic ? tE : tJ)) * dt * amp;
      for (int r = 0; r < nrec; ++r)
        for (int c = 0; c < 6; ++c)
          acc[((size_t)r * 6 + c) * nf + f] += (c < 3 ? fE : fH) * rval[r * 6 + c];
      if (vol) {
        for (int c = 0; c < 6; ++c) {
          double complex fac = (c < 3) ? fE : fH;
          double complex *vc = vol + ((size_t)c * nf + f) * nint;
          const double *Fc = st->F[c];
#pragma omp parallel for schedule(static)
          for (int k = 0; k < P->n[2]; ++k)
            for (int j = 0; j < P->n[1]; ++j)
              for (int i = 0; i < P->n[0]; ++i)
                vc[((size_t)k * P->n[1] + j) * P->n[0] + i] += fac * Fc[IDX(st, k + nbe, j + nbe, i + nbe)];
        }
      }
      if (vsa) {
        for (int q = 0; q < P->nvs; ++q) {
          long long fi = P->vs_idx[q];
          int c = (int)(fi / (long long)nint);
          long long rem = fi % (long long)nint;
          int i = (int)(rem % P->n[0]), j = (int)((rem / P->n[0]) % P->n[1]), k = (int)(rem / ((long long)P->n[0] * P->n[1]));
          vsa[(size_t)q * nf + f] += (c < 3 ? fE : fH) * st->F[c][IDX(st, k + nbe, j + nbe, i + nbe)];
        }
      }
      if (P->convergence && f == flo) {
        for (int q = 0; q < 8; ++q) {
          int ci = nbe + ((q & 1) ? P->n[0] - 1 : 0);
          int cj = nbe + ((q & 2) ? P->n[1] - 1 : 0);
          int ck = nbe + ((q & 4) ? P->n[2] - 1 : 0);
          for (int c = 0; c < 6; ++c) corner[q][c] += (c < 3 ? fE : fH) * st->F[c][IDX(st, ck, cj, ci)];
        }
      }
    }
    orc_curl_E(st, P->pml);
    /* magnetic source: mu dH/dt = -(curl E + M) (Eq. 5, time domain) */
    if (P->inject && P->magnetic) {
      for (int q = 0; q < npt * 3; ++q) {
        if (!jw[q]) continue;
        const int c = q % 3;
        for (int q3 = 0; q3 < m; ++q3)
          for (int q2 = 0; q2 < m; ++q2)
            for (int q1 = 0; q1 < m; ++q1)
              st->C[c][IDX(st, sst[q].start[2] + q3, sst[q].start[1] + q2, sst[q].start[0] + q1)]
                  += amp * jw[q][(q3 * m + q2) * m + q1];
      }
    }
    orc_update_H(st, dt);
    if (P->airwave) orc_airwave_H(st);
    if (P->convergence && it > 0 && it % 100 == 0) {
      /* converged when, at every corner, the change since the last check is at
       * most 1e-5 of the current value (and that value is nonzero). */
      int ok = 1;
      for (int q = 0; q < 8; ++q) {
        double dn = 0, un = 0;
        for (int c = 0; c < 6; ++c) {
          dn += pow(cabs(corner[q][c] - corner_prev[q][c]), 2);
          un += pow(cabs(corner[q][c]), 2);
        }
        if (!(un > 0) || sqrt(dn) > 1e-5 * sqrt(un)) ok = 0;
      }
      memcpy(corner_prev, corner, sizeof(corner));
      if (ok) { nt_run = it + 1; break; }
    }
    if (P->convergence && it == 0) memcpy(corner_prev, corner, sizeof(corner));
  }

  /* Green's functions (Eq. 7): G^EE = sqrt(-i omega / (2 omega0)) E'/J',
   * G^HE = H'/J', principal branch sqrt(omega/(2 omega0)) e^{-i pi/4}. */
  for (int f = 0; f < nf; ++f) {
    double complex sE = sqrt(2.0 * M_PI * P->freqs[f] / (2.0 * P->omega0)) * cexp(-I * M_PI / 4.0);
    if (P->jhat) { P->jhat[2 * f] = creal(jh[f]); P->jhat[2 * f + 1] = cimag(jh[f]); }
    for (int r = 0; r < nrec; ++r)
      for (int c = 0; c < 6; ++c) {
        size_t o = ((size_t)r * 6 + c) * nf + f;
        double complex g = orc_norm(c, sE, P->magnetic) * acc[o] / jh[f];
        if (P->rec_G) { P->rec_G[2 * o] = creal(g); P->rec_G[2 * o + 1] = cimag(g); }
        if (P->rec_acc) { P->rec_acc[2 * o] = creal(acc[o]); P->rec_acc[2 * o + 1] = cimag(acc[o]); }
      }
    if (vsa && P->vs_G)
      for (int q = 0; q < P->nvs; ++q) {
        int c = (int)(P->vs_idx[q] / (long long)nint);
        double complex g = orc_norm(c, sE, P->magnetic) * vsa[(size_t)q * nf + f] / jh[f];
        P->vs_G[2 * ((size_t)q * nf + f)] = creal(g);
        P->vs_G[2 * ((size_t)q * nf + f) + 1] = cimag(g);
      }
    if (vol && P->vol_G)
      for (int c = 0; c < 6; ++c) {
        double complex fac = orc_norm(c, sE, P->magnetic) / jh[f];
        double complex *vc = vol + ((size_t)c * nf + f) * nint;
        double *out = P->vol_G + 2 * ((size_t)c * nf + f) * nint;
        for (size_t q = 0; q < nint; ++q) {
          double complex g = fac * vc[q];
          out[2 * q] = creal(g); out[2 * q + 1] = cimag(g);
        }
      }
  }
  if (P->final_fields)
    for (int c = 0; c < 6; ++c) memcpy(P->final_fields + c * st->ncell, st->F[c], sizeof(double) * st->ncell);
  if (P->info) { P->info[0] = dt; P->info[1] = vmax; P->info[2] = nt_run; P->info[3] = eta; }

  free(vsa); free(vol); free(acc); free(jh); free(wp); free(rst); free(rval);
  for (int q = 0; q < npt * 3; ++q) free(jw[q]);
  free(sst);
  orc_state_free(st);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode derivative of the forward map sigma -> G (test reference for  */
/* the gradient).                                                            */
/* ------------------------------------------------------------------------ */
/* The paper computes no gradient (its Discussion leaves inversion for later);
 * this is the exact discrete adjoint of the loop of orc_forward: every linear
 * step transposed, the steps taken in reverse order.  Given a cotangent v
 * ([nrec][6][nfreq] complex) it returns
 *     grad = d/d sigma  Re( sum_{r,c,f} conj(v) G )      ([3][n3][n2][n1]),
 * the derivative with respect to the interior staggered conductivity, pads
 * included through the edge replication.  dt, nt and the CPML coefficients
 * follow from survey constants (sigma_min must be given, > 0), so the map is
 * differentiated with them fixed.  sigma enters only through dt/eps:
 *     E^{n+1} = E^n + ie (curl H - J),  ie = 2 omega0 dt / sigma,
 * hence dL/d sigma = - sum_n lambda_E^{n+1} (E^{n+1} - E^n) / sigma, with
 * lambda_E^{n+1} the adjoint of E^{n+1}.  Forward states are recomputed from
 * checkpoints taken every ckpt_every steps. */

/* Transposes of D- and D+ at sample (i,j,k): G[tap] += w[q] g. */
static void orc_dm_T(const orc_state *st, int a, double *G, int i, int j, int k, double g)
{
  int r = st->rd, m = 2 * r;
  int c = (a == 0) ? i : (a == 1 ? j : k);
  const double *w = &st->ax[a].cm[(size_t)c * m];
  for (int q = 0; q < m; ++q) {
    int ii = i, jj = j, kk = k;
    if (a == 0) ii = i - r + q; else if (a == 1) jj = j - r + q; else kk = k - r + q;
    G[IDX(st, kk, jj, ii)] += w[q] * g;
  }
}
static void orc_dp_T(const orc_state *st, int a, double *G, int i, int j, int k, double g)
{
  int r = st->rd, m = 2 * r;
  int c = (a == 0) ? i : (a == 1 ? j : k);
  const double *w = &st->ax[a].cp[(size_t)c * m];
  for (int q = 0; q < m; ++q) {
    int ii = i, jj = j, kk = k;
    if (a == 0) ii = i - r + 1 + q; else if (a == 1) jj = j - r + 1 + q; else kk = k - r + 1 + q;
    G[IDX(st, kk, jj, ii)] += w[q] * g;
  }
}

/* Transpose of the CPML step  psi' = b psi + a t,  d = t + psi'.  Given the
 * adjoint gd of d, and in mu[idx] the adjoint of psi' (from later steps),
 * return the adjoint of t and leave in mu[idx] the adjoint of the old psi. */
static double orc_pml_T(const orc_state *st, int pml, int a, int half, int c, double *mu,
                        size_t idx, double gd)
{
  if (!pml) return gd;
  int s = half ? st->ax[a].slabh[c] : st->ax[a].slab[c];
  if (s < 0) return gd;
  double aa = half ? st->ax[a].pa_h[s] : st->ax[a].pa_i[s];
  double bb = half ? st->ax[a].pb_h[s] : st->ax[a].pb_i[s];
  double gpsi = gd + mu[idx];
  mu[idx] = bb * gpsi;
  return gd + aa * gpsi;
}

/* Transpose of curl H + E update: lamH += (curl H)^T (ie lamE), CPML memory
 * adjoints muE[0..5] updated.  Serial: the transposed stencils scatter. */
static void orc_adj_E(orc_state *st, int pml, double *const *lamE, double *const *lamH, double *const *muE)
{
  for (int c = 0; c < 3; ++c) {
    int p = (c + 1) % 3, q = (c + 2) % 3, lo[3], hi[3];
    lo[c] = 0; hi[c] = st->np[c] - 2;
    orc_range_Dm(st, p, &lo[p], &hi[p]);
    orc_range_Dm(st, q, &lo[q], &hi[q]);
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t id = IDX(st, k, j, i);
          int cc[3] = {i, j, k};
          double g = st->ie[c][id] * lamE[c][id];          /* adjoint of curl H - J */
          double tp = orc_pml_T(st, pml, p, 0, cc[p], muE[2 * c], id, g);
          double tq = orc_pml_T(st, pml, q, 0, cc[q], muE[2 * c + 1], id, -g);
          orc_dm_T(st, p, lamH[q], i, j, k, tp);            /* D_p H_q */
          orc_dm_T(st, q, lamH[p], i, j, k, tq);            /* D_q H_p */
        }
  }
}

/* Transpose of curl E + H update: lamE += (curl E)^T (-dt/mu0 lamH), CPML
 * memory adjoints muH[0..5] updated. */
static void orc_adj_H(orc_state *st, int pml, double dt, double *const *lamE, double *const *lamH,
                      double *const *muH)
{
  double f = dt / ORC_MU0;
  for (int c = 0; c < 3; ++c) {
    int p = (c + 1) % 3, q = (c + 2) % 3, lo[3], hi[3];
    lo[c] = 0; hi[c] = st->np[c] - 1;
    orc_range_Dp(st, p, &lo[p], &hi[p]);
    orc_range_Dp(st, q, &lo[q], &hi[q]);
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          size_t id = IDX(st, k, j, i);
          int cc[3] = {i, j, k};
          double g = -f * lamH[c][id];                      /* adjoint of curl E */
          double tp = orc_pml_T(st, pml, p, 1, cc[p], muH[2 * c], id, g);
          double tq = orc_pml_T(st, pml, q, 1, cc[q], muH[2 * c + 1], id, -g);
          orc_dp_T(st, p, lamE[q], i, j, k, tp);            /* D_p E_q */
          orc_dp_T(st, q, lamE[p], i, j, k, tq);            /* D_q E_p */
        }
  }
}

/* Transpose of the receiver interpolation: F[nodes] += w g. */
static void orc_sample_T(const orc_state *st, double *F, const orc_stencil *s, double g)
{
  int m = 2 * st->rd;
  for (int c = 0; c < m; ++c)
    for (int b = 0; b < m; ++b)
      for (int a = 0; a < m; ++a)
        F[IDX(st, s->start[2] + c, s->start[1] + b, s->start[0] + a)] +=
            s->w[2][c] * s->w[1][b] * s->w[0][a] * g;
}

/* One forward leapfrog step without the DTFT (curl H, source, E, curl E, H). */
static void orc_step(orc_state *st, int pml, double dt, double amp, double *const *jw, const orc_stencil *sst)
{
  int m = 2 * st->rd;
  orc_curl_H(st, pml);
  for (int c = 0; c < 3; ++c) {
    if (!jw[c]) continue;
    for (int q3 = 0; q3 < m; ++q3)
      for (int q2 = 0; q2 < m; ++q2)
        for (int q1 = 0; q1 < m; ++q1)
          st->C[c][IDX(st, sst[c].start[2] + q3, sst[c].start[1] + q2, sst[c].start[0] + q1)]
              -= amp * jw[c][(q3 * m + q2) * m + q1];
  }
  orc_update_E(st);
  orc_curl_E(st, pml);
  orc_update_H(st, dt);
}

int orc_vjp(orc_problem *P, const double *v, double *grad, int ckpt_every)
{
  orc_state S, *st = &S;
  memset(st, 0, sizeof(S));
  int rd = P->rd, nb = P->nb, ne = P->ne, code = ORC_OK;
  if (rd < 1 || rd > 4 || nb < rd || ne < 0 || P->nt < 0 || P->omega0 <= 0 || !(P->sigma_min > 0) ||
      ckpt_every < 1 || !v || !grad || P->magnetic || P->src_length > 0)
    return ORC_EINVAL;
  st->rd = rd;
  for (int a = 0; a < 3; ++a) {
    code = orc_axis_nodes(&st->ax[a], P->n[a], P->x[a], rd, nb, ne);
    if (code) { orc_state_free(st); return code; }
    orc_axis_fd(&st->ax[a]);
    st->np[a] = st->ax[a].npad;
  }
  st->ncell = (size_t)st->np[0] * st->np[1] * st->np[2];
  size_t nint = (size_t)P->n[0] * P->n[1] * P->n[2], nc = st->ncell;
  for (size_t q = 0; q < 3 * nint; ++q)
    if (!(P->sigma[q] > 0) || !isfinite(P->sigma[q])) { orc_state_free(st); return ORC_EINVAL; }
  /* dt and CPML exactly as orc_forward with the given sigma_min */
  double vmax = sqrt(2.0 * P->omega0 / (ORC_MU0 * P->sigma_min));
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) { double dm = orc_axis_dmax(&st->ax[a]); d2 += dm * dm; }
  double dt = (P->dt > 0) ? P->dt : 0.99 / (0.5 * vmax * sqrt(d2));
  for (int a = 0; a < 3; ++a) orc_axis_cpml(&st->ax[a], vmax, P->fmax, dt);
  int pml = P->pml, nt = P->nt, m = 2 * rd, nbe = nb + ne;
  for (int c = 0; c < 6; ++c) st->F[c] = calloc(nc, sizeof(double));
  for (int c = 0; c < 3; ++c) { st->C[c] = calloc(nc, sizeof(double)); st->ie[c] = calloc(nc, sizeof(double)); }
  for (int c = 0; c < 12; ++c) st->psi[c] = pml ? calloc(nc, sizeof(double)) : NULL;
  for (int c = 0; c < 3; ++c) {
    const double *sg = P->sigma + c * nint;
    for (int k = 0; k < st->np[2]; ++k)
      for (int j = 0; j < st->np[1]; ++j)
        for (int i = 0; i < st->np[0]; ++i) {
          double s = sg[((size_t)orc_clampi(k - nbe, 0, P->n[2] - 1) * P->n[1] + orc_clampi(j - nbe, 0, P->n[1] - 1)) *
                            P->n[0] + orc_clampi(i - nbe, 0, P->n[0] - 1)];
          st->ie[c][IDX(st, k, j, i)] = 2.0 * P->omega0 * dt / s;
        }
  }
  /* source and receiver stencils, as in orc_forward */
  double dir[3] = {cos(P->dip) * cos(P->az), cos(P->dip) * sin(P->az), sin(P->dip)};
  orc_stencil sst[3];
  double *jw[3] = {NULL, NULL, NULL};
  for (int c = 0; c < 3 && P->inject; ++c) {
    if (dir[c] == 0.0) continue;
    for (int a = 0; a < 3 && !code; ++a)
      code = orc_locate_axis(&st->ax[a], ORC_HALF[c][a], P->src[a], &sst[c].start[a], sst[c].w[a]);
    if (code) break;
    jw[c] = malloc(sizeof(double) * m * m * m);
    for (int q3 = 0; q3 < m; ++q3)
      for (int q2 = 0; q2 < m; ++q2)
        for (int q1 = 0; q1 < m; ++q1) {
          int id3[3] = {sst[c].start[0] + q1, sst[c].start[1] + q2, sst[c].start[2] + q3};
          double V = 1.0;
          for (int a = 0; a < 3; ++a) {
            const orc_axis *ax = &st->ax[a];
            V *= ORC_HALF[c][a] ? (ax->X[id3[a] + 1] - ax->X[id3[a]]) : (ax->Xh[id3[a]] - ax->Xh[id3[a] - 1]);
          }
          jw[c][(q3 * m + q2) * m + q1] = dir[c] * sst[c].w[0][q1] * sst[c].w[1][q2] * sst[c].w[2][q3] / V;
        }
  }
  int nrec = P->nrec, nf = P->nfreq;
  orc_stencil *rst = calloc((size_t)(nrec > 0 ? nrec : 1) * 6, sizeof(orc_stencil));
  for (int r = 0; r < nrec && !code; ++r)
    for (int c = 0; c < 6 && !code; ++c)
      for (int a = 0; a < 3 && !code; ++a)
        code = orc_locate_axis(&st->ax[a], ORC_HALF[c][a], P->rec[3 * r + a], &rst[r * 6 + c].start[a],
                               rst[r * 6 + c].w[a]);
  if (code) { free(rst); for (int c = 0; c < 3; ++c) free(jw[c]); orc_state_free(st); return code; }

  /* source spectrum J' and the weights c_{r,c,f} = conj(v) s_c / J' of Eq. 7:
   * dL/du_{r,c,n} = Re( sum_f c_{r,c,f} e^{i w' t_n} dt ) */
  double complex *wp = malloc(sizeof(double complex) * (nf > 0 ? nf : 1));
  double complex *jh = calloc(nf > 0 ? nf : 1, sizeof(double complex));
  for (int f = 0; f < nf; ++f) wp[f] = (1.0 + I) * sqrt(2.0 * M_PI * P->freqs[f] * P->omega0);
  for (int n = 0; n < nt; ++n)
    for (int f = 0; f < nf; ++f)
      jh[f] += cexp(I * wp[f] * ((n + 0.5) * dt)) * dt * P->moment * orc_wavelet((n + 0.5) * dt, P->fmax);
  double complex *cw = calloc((size_t)(nrec > 0 ? nrec : 1) * 6 * (nf > 0 ? nf : 1), sizeof(double complex));
  for (int f = 0; f < nf; ++f) {
    double complex sE = sqrt(2.0 * M_PI * P->freqs[f] / (2.0 * P->omega0)) * cexp(-I * M_PI / 4.0);
    for (int r = 0; r < nrec; ++r)
      for (int c = 0; c < 6; ++c) {
        size_t o = ((size_t)r * 6 + c) * nf + f;
        double complex vv = v[2 * o] + I * v[2 * o + 1];
        cw[o] = conj(vv) * (c < 3 ? sE : 1.0) / jh[f];
      }
  }

  /* forward sweep: checkpoints of the whole state before steps 0, K, 2K, ... */
  int K = ckpt_every, nck = (nt + K - 1) / K;
  int nstate = pml ? 18 : 6;
  double *ck = malloc(sizeof(double) * (size_t)(nck > 0 ? nck : 1) * nstate * nc);
  double *Eh = malloc(sizeof(double) * (size_t)(K + 1) * 3 * nc);
  double *lam[6], *mu[12], *gpad[3];
  for (int c = 0; c < 6; ++c) lam[c] = calloc(nc, sizeof(double));
  for (int c = 0; c < 12; ++c) mu[c] = pml ? calloc(nc, sizeof(double)) : NULL;
  for (int c = 0; c < 3; ++c) gpad[c] = calloc(nc, sizeof(double));
  if (!ck || !Eh) code = ORC_ENOMEM;
  for (int it = 0; it < nt && !code; ++it) {
    if (it % K == 0) {
      double *dst = ck + (size_t)(it / K) * nstate * nc;
      for (int c = 0; c < 6; ++c) memcpy(dst + c * nc, st->F[c], sizeof(double) * nc);
      for (int c = 0; c < 12 && pml; ++c) memcpy(dst + (6 + c) * nc, st->psi[c], sizeof(double) * nc);
    }
    orc_step(st, pml, dt, P->moment * orc_wavelet((it + 0.5) * dt, P->fmax), jw, sst);
  }

  /* reverse sweep, one checkpoint segment at a time */
  for (int s = nck - 1; s >= 0 && !code; --s) {
    int it0 = s * K, it1 = (it0 + K < nt) ? it0 + K : nt;
    const double *src = ck + (size_t)s * nstate * nc;
    for (int c = 0; c < 6; ++c) memcpy(st->F[c], src + c * nc, sizeof(double) * nc);
    for (int c = 0; c < 12 && pml; ++c) memcpy(st->psi[c], src + (6 + c) * nc, sizeof(double) * nc);
    for (int it = it0; it < it1; ++it) {
      for (int c = 0; c < 3; ++c) memcpy(Eh + ((size_t)(it - it0) * 3 + c) * nc, st->F[c], sizeof(double) * nc);
      orc_step(st, pml, dt, P->moment * orc_wavelet((it + 0.5) * dt, P->fmax), jw, sst);
    }
    for (int c = 0; c < 3; ++c) memcpy(Eh + ((size_t)(it1 - it0) * 3 + c) * nc, st->F[c], sizeof(double) * nc);
    for (int it = it1 - 1; it >= it0; --it) {
      /* H update of step it: H^{it+3/2} = H^{it+1/2} - dt/mu0 curl E^{it+1} */
      orc_adj_H(st, pml, dt, lam, lam + 3, mu + 6);
      /* receiver DTFT of E^{it+1} (label (it+1) dt) and H^{it+1/2} ((it+1/2) dt) */
      for (int r = 0; r < nrec; ++r)
        for (int c = 0; c < 6; ++c) {
          double t = (c < 3) ? (it + 1.0) * dt : (it + 0.5) * dt, g = 0.0;
          for (int f = 0; f < nf; ++f) g += creal(cw[((size_t)r * 6 + c) * nf + f] * cexp(I * wp[f] * t) * dt);
          orc_sample_T(st, lam[c], &rst[r * 6 + c], g);
        }
      /* gradient: dL/dsigma += - lambda_E^{it+1} (E^{it+1} - E^it) / sigma,
       * with sigma = 2 omega0 dt / ie on the padded grid */
      const double *E0 = Eh + (size_t)(it - it0) * 3 * nc, *E1 = Eh + (size_t)(it - it0 + 1) * 3 * nc;
      for (int c = 0; c < 3; ++c)
        for (size_t id = 0; id < nc; ++id) {
          double dE = E1[c * nc + id] - E0[c * nc + id];
          if (dE != 0.0) gpad[c][id] -= lam[c][id] * dE * st->ie[c][id] / (2.0 * P->omega0 * dt);
        }
      /* E update of step it */
      orc_adj_E(st, pml, lam, lam + 3, mu);
    }
  }
  /* fold the padded gradient onto the interior samples it replicates */
  if (!code) {
    memset(grad, 0, sizeof(double) * 3 * nint);
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < st->np[2]; ++k)
        for (int j = 0; j < st->np[1]; ++j)
          for (int i = 0; i < st->np[0]; ++i) {
            size_t o = ((size_t)orc_clampi(k - nbe, 0, P->n[2] - 1) * P->n[1] + orc_clampi(j - nbe, 0, P->n[1] - 1)) *
                           P->n[0] + orc_clampi(i - nbe, 0, P->n[0] - 1);
            grad[c * nint + o] += gpad[c][IDX(st, k, j, i)];
          }
  }
  for (int c = 0; c < 6; ++c) free(lam[c]);
  for (int c = 0; c < 12; ++c) free(mu[c]);
  for (int c = 0; c < 3; ++c) { free(gpad[c]); free(jw[c]); }
  free(ck); free(Eh); free(cw); free(jh); free(wp); free(rst);
  orc_state_free(st);
  return code;
}

/* ------------------------------------------------------------------------
 * Conductivity model on the staggered grid (Sec. 3.6).
 *
 * Cells lie between adjacent interior nodes ([n3-1][n2-1][n1-1], x fastest)
 * and carry sigma_h and sigma_v.  The staggered sigma_cc of E_c at a sample
 * is the mean over the cells around its edge, each weighted by its face area
 * across the edge: along the two axes a, b across the edge, node j touches
 * cells j-1 and j (clamped to the model, so an edge on a face of the model
 * names its one cell twice); along the edge's own axis the sample lies in
 * cell min(i, n-2).  sigma_h feeds sigma_xx and sigma_yy, sigma_v sigma_zz.
 * orc_stagger applies this sparse map, orc_stagger_T its transpose, both
 * through the (cell, weight) list of orc_stagger_terms.
 * ------------------------------------------------------------------------ */
static void orc_cell_pair(int j, int n, int c[2])
{
  c[0] = orc_clampi(j - 1, 0, n - 2);
  c[1] = orc_clampi(j, 0, n - 2);
}

/* The four (cell, weight) terms of staggered sample (comp, idx); weights sum to 1. */
static void orc_stagger_terms(const int n[3], double *const w[3], int comp, const int idx[3], size_t cell[4],
                              double wt[4])
{
  int a = comp == 0 ? 1 : 0, b = comp == 2 ? 1 : 2, ca[2], cb[2], cc[3];
  orc_cell_pair(idx[a], n[a], ca);
  orc_cell_pair(idx[b], n[b], cb);
  cc[comp] = orc_clampi(idx[comp], 0, n[comp] - 2);
  double tot = 0.0;
  for (int q = 0; q < 4; ++q) {
    cc[a] = ca[q & 1];
    cc[b] = cb[q >> 1];
    wt[q] = w[a][cc[a]] * w[b][cc[b]];
    tot += wt[q];
    cell[q] = ((size_t)cc[2] * (n[1] - 1) + cc[1]) * (n[0] - 1) + cc[0];
  }
  for (int q = 0; q < 4; ++q) wt[q] /= tot;
}

static int orc_widths(const int n[3], const double *const x[3], double *w[3])
{
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 2) return ORC_EINVAL;
    w[a] = malloc(sizeof(double) * (n[a] - 1));
    for (int c = 0; c + 1 < n[a]; ++c) w[a][c] = x[a][c + 1] - x[a][c];
  }
  return ORC_OK;
}

/* out[3][n3][n2][n1] = staggered sigma from sh, sv [n3-1][n2-1][n1-1]. */
int orc_stagger(const int n[3], const double *const x[3], const double *sh, const double *sv, double *out)
{
  double *w[3] = {0, 0, 0};
  int code = orc_widths(n, x, w);
  if (!code) {
    size_t per = (size_t)n[0] * n[1] * n[2];
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            int idx[3] = {i, j, k};
            size_t cell[4];
            double wt[4], s = 0.0;
            orc_stagger_terms(n, w, c, idx, cell, wt);
            for (int q = 0; q < 4; ++q) s += wt[q] * (c == 2 ? sv : sh)[cell[q]];
            out[c * per + ((size_t)k * n[1] + j) * n[0] + i] = s;
          }
  }
  for (int a = 0; a < 3; ++a) free(w[a]);
  return code;
}

/* Transpose: gh, gv [n3-1][n2-1][n1-1] = S^T g, g [3][n3][n2][n1] (overwritten). */
int orc_stagger_T(const int n[3], const double *const x[3], const double *g, double *gh, double *gv)
{
  double *w[3] = {0, 0, 0};
  int code = orc_widths(n, x, w);
  if (!code) {
    size_t per = (size_t)n[0] * n[1] * n[2], ncell = (size_t)(n[0] - 1) * (n[1] - 1) * (n[2] - 1);
    memset(gh, 0, sizeof(double) * ncell);
    memset(gv, 0, sizeof(double) * ncell);
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            int idx[3] = {i, j, k};
            size_t cell[4];
            double wt[4], gs = g[c * per + ((size_t)k * n[1] + j) * n[0] + i];
            orc_stagger_terms(n, w, c, idx, cell, wt);
            for (int q = 0; q < 4; ++q) (c == 2 ? gv : gh)[cell[q]] += wt[q] * gs;
          }
  }
  for (int a = 0; a < 3; ++a) free(w[a]);
  return code;
}
