// Conductivity model on the staggered grid (Sec. 3.6): the staggered
// conductivities sigma_xx, sigma_yy, sigma_zz the solver consumes, from
// cell-centred horizontal and vertical conductivities, and the transpose of
// that linear map, which carries a gradient with respect to the staggered
// samples back to the cells.
//
// The cells are those between adjacent interior nodes, [n3-1][n2-1][n1-1].
// E_x sits on the edge (x_{i+1/2}, y_j, z_k) shared by the (up to) four cells
// around it in y and z; sigma_xx there is the mean of their sigma_h weighted
// by the cells' y-z face areas dy * dz.  sigma_yy likewise over x and z, and
// sigma_zz averages sigma_v over the four cells around the edge in x and y.
// Along the edge's own axis the sample belongs to cell min(i, n-2) (the last
// half node lies beyond the last interior node); across it, node j touches
// cells j-1 and j clamped to [0, n-2], so an edge on the model's faces
// averages the one cell it touches.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "emm_internal.h"

namespace emm {
namespace {

// Interior cell widths per axis: w[ax][c] = x_{c+1} - x_c, c in [0, n-1).
struct Widths {
  const double *w[3];
  int n[3];
};

__device__ __forceinline__ int cell_lo(int j, int n) { return min(max(j - 1, 0), n - 2); }
__device__ __forceinline__ int cell_hi(int j, int n) { return min(j, n - 2); }

// One thread per staggered sample of [3][n3][n2][n1].
__global__ void k_stagger(const Widths W, const double *sh, const double *sv, float *sig) {
  const int n1 = W.n[0], n2 = W.n[1], n3 = W.n[2];
  const size_t per = static_cast<size_t>(n1) * n2 * n3;
  const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= 3 * per) return;
  const int c = static_cast<int>(t / per);
  const size_t r = t % per;
  const int i = static_cast<int>(r % n1), j = static_cast<int>((r / n1) % n2), k = static_cast<int>(r / (static_cast<size_t>(n1) * n2));
  const int idx[3] = {i, j, k};
  // the two axes across the edge (a, b) and the one along it (c)
  const int a = c == 0 ? 1 : 0, b = c == 2 ? 1 : 2;
  const double *field = c == 2 ? sv : sh;
  int cell[3];
  cell[c] = min(idx[c], W.n[c] - 2);
  const int ca[2] = {cell_lo(idx[a], W.n[a]), cell_hi(idx[a], W.n[a])};
  const int cb[2] = {cell_lo(idx[b], W.n[b]), cell_hi(idx[b], W.n[b])};
  double s = 0.0, w = 0.0;
  for (int pb = 0; pb < 2; ++pb)
    for (int pa = 0; pa < 2; ++pa) {
      cell[a] = ca[pa];
      cell[b] = cb[pb];
      const double ww = W.w[b][cb[pb]] * W.w[a][ca[pa]];
      s += ww * field[(static_cast<size_t>(cell[2]) * (n2 - 1) + cell[1]) * (n1 - 1) + cell[0]];
      w += ww;
    }
  sig[t] = static_cast<float>(s / w);
}

// Weight of cell `cell` in the across-edge pair of node j along an axis of n
// nodes (the raw width; a clamped pair names the same cell twice), and the
// pair's total width.
__device__ __forceinline__ double pair_weight(const double *w, int n, int j, int cell, double *total) {
  const int lo = cell_lo(j, n), hi = cell_hi(j, n);
  *total = w[lo] + w[hi];
  return (lo == cell ? w[lo] : 0.0) + (hi == cell ? w[hi] : 0.0);
}

// One thread per cell: gather the weighted gradients of every staggered
// sample whose mean contains the cell, and add them to grad_h / grad_v.
__global__ void k_stagger_adjoint(const Widths W, const double *g, double *gh, double *gv) {
  const int n1 = W.n[0], n2 = W.n[1], n3 = W.n[2];
  const size_t ncell = static_cast<size_t>(n1 - 1) * (n2 - 1) * (n3 - 1);
  const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= ncell) return;
  const int cx = static_cast<int>(t % (n1 - 1)), cy = static_cast<int>((t / (n1 - 1)) % (n2 - 1)),
            cz = static_cast<int>(t / (static_cast<size_t>(n1 - 1) * (n2 - 1)));
  const int cel[3] = {cx, cy, cz};
  const size_t per = static_cast<size_t>(n1) * n2 * n3;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < 3; ++c) {
    const int a = c == 0 ? 1 : 0, b = c == 2 ? 1 : 2;
    // samples along the edge axis owned by this cell: the cell's own index,
    // and the last half node when this is the last cell
    const int own_n = cel[c] == W.n[c] - 2 ? 2 : 1;
    for (int o = 0; o < own_n; ++o) {
      const int ic = cel[c] + o;
      // across the edge, nodes cel and cel + 1 are the ones whose pair holds the cell
      for (int qb = 0; qb < 2; ++qb) {
        double tb;
        const int jb = cel[b] + qb;
        const double wb = pair_weight(W.w[b], W.n[b], jb, cel[b], &tb);
        for (int qa = 0; qa < 2; ++qa) {
          double ta;
          const int ja = cel[a] + qa;
          const double wa = pair_weight(W.w[a], W.n[a], ja, cel[a], &ta);
          int id[3];
          id[c] = ic;
          id[a] = ja;
          id[b] = jb;
          const size_t s = static_cast<size_t>(c) * per + (static_cast<size_t>(id[2]) * n2 + id[1]) * n1 + id[0];
          acc[c] += g[s] * (wa * wb) / (ta * tb);
        }
      }
    }
  }
  gh[t] += acc[0] + acc[1];
  gv[t] += acc[2];
}

size_t widths_bytes(const emm_grid *g) {
  size_t b = 0;
  for (int a = 0; a < 3; ++a) b += static_cast<size_t>(g->ax[a].n - 1) * sizeof(double);
  return b;
}

// Copies the interior cell widths into ws and points W at them.
int load_widths(const emm_grid *g, void *ws, size_t ws_bytes, cudaStream_t cs, Widths *W) {
  if (!ws || ws_bytes < widths_bytes(g) || (reinterpret_cast<uintptr_t>(ws) % 8) != 0) return EMM_EWORKSPACE;
  const int nbe = g->nb + g->ne;
  std::vector<double> h;
  for (int a = 0; a < 3; ++a) {
    W->n[a] = g->ax[a].n;
    for (int c = 0; c + 1 < g->ax[a].n; ++c) h.push_back(g->ax[a].X[nbe + c + 1] - g->ax[a].X[nbe + c]);
  }
  double *d = static_cast<double *>(ws);
  size_t off = 0;
  for (int a = 0; a < 3; ++a) {
    W->w[a] = d + off;
    off += static_cast<size_t>(g->ax[a].n - 1);
  }
  // pageable source: the copy has taken the data when it returns
  return cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, cs) == cudaSuccess
             ? EMM_OK
             : EMM_ECUDA;
}

}  // namespace
}  // namespace emm

extern "C" {

int emm_stagger_workspace_size(const emm_grid *g, size_t *bytes) {
  if (!g || !bytes) return EMM_EINVAL;
  *bytes = emm::widths_bytes(g);
  return EMM_OK;
}

int emm_stagger_sigma(const emm_grid *g, const double *sigma_h, const double *sigma_v, void *ws, size_t ws_bytes,
                      float *sigma, emm_stream stream) {
  if (!g || !sigma_h || !sigma_v || !sigma) return EMM_EINVAL;
  const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::Widths W{};
  const int st = emm::load_widths(g, ws, ws_bytes, cs, &W);
  if (st != EMM_OK) return st;
  const size_t n = 3 * static_cast<size_t>(W.n[0]) * W.n[1] * W.n[2];
  emm::k_stagger<<<static_cast<unsigned>((n + 255) / 256), 256, 0, cs>>>(W, sigma_h, sigma_v, sigma);
  return cudaGetLastError() == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

int emm_stagger_sigma_adjoint(const emm_grid *g, const double *grad, void *ws, size_t ws_bytes, double *grad_h,
                              double *grad_v, emm_stream stream) {
  if (!g || !grad || !grad_h || !grad_v) return EMM_EINVAL;
  const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::Widths W{};
  const int st = emm::load_widths(g, ws, ws_bytes, cs, &W);
  if (st != EMM_OK) return st;
  const size_t n = static_cast<size_t>(W.n[0] - 1) * (W.n[1] - 1) * (W.n[2] - 1);
  emm::k_stagger_adjoint<<<static_cast<unsigned>((n + 255) / 256), 256, 0, cs>>>(W, grad, grad_h, grad_v);
  return cudaGetLastError() == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

}  // extern "C"
