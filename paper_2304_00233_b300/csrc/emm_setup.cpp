// emm_setup.cpp -- host side of libemm: grid padding, finite-difference rows,
// CPML coefficients, the stability time step, and source/receiver stencils.
//
// Everything here runs once per grid or per forward call, in FP64 (Sec. 4.1:
// all pre-computation happens on the host before the time stepping moves to
// the GPU).  The FD rows are row 1 and the interpolation weights row 0 of
// [V^T]^{-1} (Sec. 3.1 Eq. 9-11); they are evaluated here from the closed
// form of the Lagrange basis and its derivative, which is that inverse's
// definition (p(x) = sum_j L_j(x) f_j, p'(x) = sum_j L_j'(x) f_j).
#include <cmath>
#include <cstring>
#include <new>

#include "emm_internal.h"

using emm::Axis;

namespace {

// Lagrange basis at x for knots t[0..m-1]: w0[j] = L_j(x), w1[j] = L_j'(x).
void lagrange_rows(int m, const double *t, double x, double *w0, double *w1) {
  for (int j = 0; j < m; ++j) {
    double denom = 1.0;
    for (int l = 0; l < m; ++l)
      if (l != j) denom *= (t[j] - t[l]);
    double val = 1.0;
    for (int l = 0; l < m; ++l)
      if (l != j) val *= (x - t[l]);
    double der = 0.0;  // d/dx prod_{l != j} (x - t_l) = sum_l prod_{q != j,l} (x - t_q)
    for (int l = 0; l < m; ++l) {
      if (l == j) continue;
      double prod = 1.0;
      for (int q = 0; q < m; ++q)
        if (q != j && q != l) prod *= (x - t[q]);
      der += prod;
    }
    if (w0) w0[j] = val / denom;
    if (w1) w1[j] = der / denom;
  }
}

int build_axis(Axis &ax, int n, const double *x, int rd, int nb, int ne) {
  if (n < 2 || x == nullptr) return EMM_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(x[i]) || (i > 0 && !(x[i] > x[i - 1]))) return EMM_EINVAL;
  const int nbe = nb + ne, np = n + 2 * nbe, m = 2 * rd;
  ax.n = n;
  ax.npad = np;
  try {
    ax.X.assign(np + 1, 0.0);
    ax.Xh.assign(np, 0.0);
    ax.cp.assign(static_cast<size_t>(np) * m, 0.0);
    ax.cm.assign(static_cast<size_t>(np) * m, 0.0);
    ax.cp_start.assign(np, -1);
    ax.cm_start.assign(np, -1);
    ax.slab_i.assign(np, -1);
    ax.slab_h.assign(np, -1);
  } catch (const std::bad_alloc &) {
    return EMM_ENOMEM;
  }
  // pads repeat the edge spacing on each side; X[np] bounds the last half cell
  const double lo_step = x[1] - x[0], hi_step = x[n - 1] - x[n - 2];
  for (int i = 0; i < n; ++i) ax.X[nbe + i] = x[i];
  for (int k = 1; k <= nbe; ++k) ax.X[nbe - k] = x[0] - k * lo_step;
  for (int k = 1; k <= nbe + 1; ++k) ax.X[nbe + n - 1 + k] = x[n - 1] + k * hi_step;
  for (int i = 0; i < np; ++i) ax.Xh[i] = 0.5 * (ax.X[i] + ax.X[i + 1]);
  // The grid has integer samples 0..np-1 and half samples 0..np-2 (the half
  // sample past the last node is never updated).  D+ at Xh[i] needs integer
  // samples i-rd+1..i+rd; D- at X[i] needs half samples i-rd..i+rd-1.
  for (int i = rd - 1; i <= np - 1 - rd; ++i) {
    ax.cp_start[i] = i - rd + 1;
    lagrange_rows(m, &ax.X[i - rd + 1], ax.Xh[i], nullptr, &ax.cp[static_cast<size_t>(i) * m]);
  }
  for (int i = rd; i <= np - 1 - rd; ++i) {
    ax.cm_start[i] = i - rd;
    lagrange_rows(m, &ax.Xh[i - rd], ax.X[i], nullptr, &ax.cm[static_cast<size_t>(i) * m]);
  }
  // CPML slabs: nb samples of each kind per face, far face mirrored
  // (integer sample i <-> np-1-i, half sample i <-> np-2-i).
  for (int s = 0; s < nb; ++s) {
    ax.slab_i[s] = s;
    ax.slab_i[np - 1 - s] = nb + s;
    ax.slab_h[s] = s;
    ax.slab_h[np - 2 - s] = nb + s;
  }
  return EMM_OK;
}

}  // namespace

namespace emm {

double dmax_axis(const Axis &ax, int rd) {
  const int m = 2 * rd;
  double best = 0.0;
  for (int i = 0; i < ax.npad; ++i) {
    double sp = 0.0, sm = 0.0;
    for (int q = 0; q < m; ++q) {
      sp += std::fabs(ax.cp[static_cast<size_t>(i) * m + q]);
      sm += std::fabs(ax.cm[static_cast<size_t>(i) * m + q]);
    }
    best = std::fmax(best, std::fmax(sp, sm));
  }
  return best;
}

// CPML damping of Eq. 23-24 with kappa = 1.  For slab entry s the sample's
// depth xi into its layer is measured from the layer's inner face (X[nb] on
// the low side, X[np-1-nb] on the high side); L is that face's thickness.
void cpml_axis(const emm_grid *g, int axis, double vmax, double fmax, double dt, double *ab) {
  const Axis &ax = g->ax[axis];
  const int nb = g->nb, np = ax.npad;
  const double lowL = ax.X[nb] - ax.X[0];
  const double highL = ax.X[np - 1] - ax.X[np - 1 - nb];
  auto coef = [&](int s, double pos, double *a, double *b) {
    const bool low = s < nb;
    const double L = low ? lowL : highL;
    double depth = low ? (ax.X[nb] - pos) : (pos - ax.X[np - 1 - nb]);
    depth = std::fmin(std::fmax(depth, 0.0), L);
    const double u = depth / L;
    const double d = -3.0 * vmax * std::log(1.0e-3) / (2.0 * L) * u * u;
    const double alpha = M_PI * fmax * (1.0 - u);
    *b = std::exp(-(d + alpha) * dt);
    *a = (d + alpha > 0.0) ? d / (d + alpha) * (*b - 1.0) : 0.0;
  };
  for (int s = 0; s < 2 * nb; ++s) {
    const int ii = (s < nb) ? s : np - 1 - (s - nb);
    const int ih = (s < nb) ? s : np - 2 - (s - nb);
    coef(s, ax.X[ii], &ab[s], &ab[2 * nb + s]);
    coef(s, ax.Xh[ih], &ab[4 * nb + s], &ab[6 * nb + s]);
  }
}

// Stencil of a point on one axis: P = X or Xh, i = max{i : P[i] <= p}, knots
// i-rd+1 .. i+rd, all outside the CPML slabs; w = Lagrange weights at p.
int locate_axis(const emm_grid *g, int axis, int half, double p, int *start, double *w) {
  const Axis &ax = g->ax[axis];
  const int rd = g->rd, nb = g->nb, np = ax.npad;
  const double *P = half ? ax.Xh.data() : ax.X.data();
  const int last = half ? np - 2 : np - 1;   // last sample on the grid
  if (!std::isfinite(p) || !(p >= P[0])) return EMM_EOUTSIDE;
  int lo = 0, hi = last;                      // P ascending: binary search for max{i: P[i] <= p}
  if (p >= P[last]) {
    lo = last;
  } else {
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (P[mid] <= p) lo = mid; else hi = mid;
    }
  }
  const int s = lo - rd + 1;
  if (s < nb || lo + rd > np - 1 - nb) return EMM_EOUTSIDE;
  *start = s;
  lagrange_rows(2 * rd, P + s, p, w, nullptr);
  return EMM_OK;
}

}  // namespace emm

extern "C" {

int emm_make_grid(const emm_grid_desc *d, emm_grid **out) {
  if (!d || !out) return EMM_EINVAL;
  *out = nullptr;
  if (d->rd < 1 || d->rd > emm::kMaxRd || d->nb < d->rd || d->ne < 0) return EMM_EINVAL;
  emm_grid *g = new (std::nothrow) emm_grid;
  if (!g) return EMM_ENOMEM;
  g->rd = d->rd;
  g->nb = d->nb;
  g->ne = d->ne;
  for (int a = 0; a < 3; ++a) {
    const int st = build_axis(g->ax[a], d->n[a], d->x[a], d->rd, d->nb, d->ne);
    if (st != EMM_OK) {
      delete g;
      return st;
    }
  }
  *out = g;
  return EMM_OK;
}

void emm_free_grid(emm_grid *g) { delete g; }

int emm_grid_query(const emm_grid *g, emm_grid_info *info) {
  if (!g || !info) return EMM_EINVAL;
  info->cells = 1;
  for (int a = 0; a < 3; ++a) {
    info->n[a] = g->ax[a].n;
    info->npad[a] = g->ax[a].npad;
    info->cells *= static_cast<size_t>(g->ax[a].npad);
  }
  info->rd = g->rd;
  info->nb = g->nb;
  info->ne = g->ne;
  return EMM_OK;
}

int emm_grid_tables(const emm_grid *g, int axis, int kind, double *coef, int *idx) {
  if (!g || axis < 0 || axis > 2) return EMM_EINVAL;
  const Axis &ax = g->ax[axis];
  auto cpy_d = [&](const std::vector<double> &v) {
    if (coef) std::memcpy(coef, v.data(), v.size() * sizeof(double));
  };
  auto cpy_i = [&](const std::vector<int> &v) {
    if (idx) std::memcpy(idx, v.data(), v.size() * sizeof(int));
  };
  switch (kind) {
    case EMM_TAB_NODES: cpy_d(ax.X); break;
    case EMM_TAB_HALF: cpy_d(ax.Xh); break;
    case EMM_TAB_DPLUS: cpy_d(ax.cp); cpy_i(ax.cp_start); break;
    case EMM_TAB_DMINUS: cpy_d(ax.cm); cpy_i(ax.cm_start); break;
    case EMM_TAB_SLAB_INT: cpy_i(ax.slab_i); break;
    case EMM_TAB_SLAB_HALF: cpy_i(ax.slab_h); break;
    default: return EMM_EINVAL;
  }
  return EMM_OK;
}

int emm_time_step(const emm_grid *g, double sigma_min, double omega0, double *dt,
                  double *eta, double *vmax) {
  if (!g || !(sigma_min > 0.0) || !(omega0 > 0.0) || !std::isfinite(sigma_min)) return EMM_EINVAL;
  const double v = std::sqrt(2.0 * omega0 / (emm::kMu0 * sigma_min));
  double s2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double dm = emm::dmax_axis(g->ax[a], g->rd);
    s2 += dm * dm;
  }
  const double e = 0.5 * v * std::sqrt(s2);
  if (dt) *dt = 0.99 / e;
  if (eta) *eta = e;
  if (vmax) *vmax = v;
  return EMM_OK;
}

int emm_cpml_tables(const emm_grid *g, int axis, double vmax, double fmax, double dt, double *ab) {
  if (!g || !ab || axis < 0 || axis > 2 || !(vmax > 0) || !(fmax > 0) || !(dt > 0)) return EMM_EINVAL;
  emm::cpml_axis(g, axis, vmax, fmax, dt, ab);
  return EMM_OK;
}

int emm_locate(const emm_grid *g, int comp, const double pos[3], int start[3], double *w) {
  if (!g || !pos || !start || !w || comp < 0 || comp > 5) return EMM_EINVAL;
  const int m = 2 * g->rd;
  for (int a = 0; a < 3; ++a) {
    const int st = emm::locate_axis(g, a, emm::kHalf[comp][a], pos[a], &start[a], w + a * m);
    if (st != EMM_OK) return st;
  }
  return EMM_OK;
}

const char *emm_strerror(int code) {
  switch (code) {
    case EMM_OK: return "ok";
    case EMM_EINVAL: return "invalid argument";
    case EMM_ENOMEM: return "host allocation failed";
    case EMM_EOUTSIDE: return "source or receiver stencil outside the non-CPML region";
    case EMM_ECFL: return "time step exceeds the stability limit 1/eta";
    case EMM_ECUDA: return "CUDA runtime error";
    case EMM_EWORKSPACE: return "workspace too small or misaligned";
    case EMM_EDEVICE: return "device detected an invalid conductivity value";
    case EMM_ETIMEOUT: return "a bounded device-side wait ran out";
    default: return "unknown error";
  }
}

}  // extern "C"
