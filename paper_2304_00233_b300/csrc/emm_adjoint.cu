// emm_adjoint.cu -- gradient of the receiver Green's functions with respect to
// the staggered conductivity: emm_gradient_workspace_size and emm_gradient.
//
// The paper stops at the forward solver (its Discussion names inversion as
// future work).  This is the exact discrete adjoint of the time loop the
// forward kernels run: every linear step of a leapfrog step transposed and
// the steps taken in reverse order.  For a cotangent v of the Green's
// functions G (complex, [nrec][6][nfreq]) it returns
//     grad = d/d sigma Re( sum conj(v) G ),
// the vector-Jacobian product a torch.autograd.Function needs.  sigma enters
// the loop only through dt/eps (E^{n+1} = E^n + ie (curl H - J), ie = 2 omega0
// dt / sigma), so
//     dL/d sigma = - sum_n lambda_E^{n+1} (E^{n+1} - E^n) / sigma,
// lambda_E^{n+1} being the adjoint of E^{n+1}.  dt, nt and the CPML
// coefficients depend on survey constants (sigma_min, fmax), not on sigma.
//
// Schedule: a forward sweep stores the whole state (fields and CPML memory)
// every K steps; the reverse sweep, one checkpoint segment at a time,
// recomputes the segment's E snapshots and then runs the adjoint steps
// backwards.  One adjoint step, the transpose of one forward step, is three
// launches:
//   1. receivers: lambda += interpolation^T of Re(conj(v) norm f_n);
//   2. H update transposed: lambda_E += (D+)^T T_H (a TMA-fed gather), T_H
//      the per-derivative adjoints -dt/mu0 lambda_H formed with the CPML
//      memory adjoints by the previous launch 3; its epilogue forms, from the
//      final lambda_E, the gradient term g -= lambda_E (E^{n+1} - E^n) /
//      sigma (FP32 within a checkpoint segment, added into FP64 at its end)
//      and T_E = dt/eps lambda_E with the CPML;
//   3. E update transposed: lambda_H += (D-)^T T_E; its epilogue forms T_H
//      of the step before from the final lambda_H.
// Finally the padded gradient is folded onto the interior samples the pads
// replicate.  Adjoint fields are FP32 like the forward fields; the gradient
// accumulates in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "emm_internal.h"
#include "emm_tma.cuh"

namespace emm {
namespace {

constexpr int kThreads = 256;

struct AdjParams {
  int np[3], n[3], pitch, nb, rd, nbe, org[3];
  size_t plane;
  float kappa;               // dt / mu0
  float inv_2w0dt;           // 1 / (2 omega0 dt): sigma = 2 omega0 dt / ie
  const float *ie[3];
  float *lamE[3], *lamH[3];  // adjoint fields (field layout)
  float *TH[6], *TE[6];      // per-derivative adjoints of the H and the E half step (field layout)
  int *status;
  float *muE[6], *muH[6];    // adjoints of the CPML memory (psi layouts)
  int psx_hx[2], psx_wx[2], psx_far0[2];
  const float *pml[3];       // [4][2nb]: a_int, b_int, a_half, b_half
  const float *cpT[3];       // transposed D+ rows, gather form [rows][2rd]
  const float *cmT[3];       // transposed D- rows, gather form [rows][2rd]
  const float *E0[3], *E1[3];  // forward E before / after the step
  double *gpad[3];           // dL/dsigma on the padded grid (field layout)
  float *gseg[3];            // the current segment's share, FP32, flushed into gpad
  int nrec, nf;
  const int *rec_start;      // [nrec][6][3]
  const double *rec_w;       // [nrec][6][3][2rd]
  const double *cw;          // [nrec][6][nf][2]: conj(v) * norm
  const double *fE, *fH;     // [nt][nf][2]
};

__device__ __forceinline__ int slab_int(int i, int np, int nb) {
  return i < nb ? i : (i >= np - nb ? nb + np - 1 - i : -1);
}
__device__ __forceinline__ int slab_half(int i, int np, int nb) {
  return i < nb ? i : ((i >= np - 1 - nb && i <= np - 2) ? nb + np - 2 - i : -1);
}

// Cell of this thread in a 3-D launch of 32 x 8 threads per (x, y) tile and
// one grid z layer per plane; false outside the padded grid.
__device__ __forceinline__ bool cell3(const AdjParams &a, int *idx) {
  idx[0] = blockIdx.x * 32 + threadIdx.x;
  idx[1] = blockIdx.y * 8 + threadIdx.y;
  idx[2] = blockIdx.z;
  return idx[0] < a.np[0] && idx[1] < a.np[1];
}
__device__ __forceinline__ size_t fid(const AdjParams &a, int i, int j, int k) {
  return static_cast<size_t>(k) * a.plane + static_cast<size_t>(j) * a.pitch + i;
}

// The per-derivative adjoint of a forward term, T = g (+ the transposed CPML
// step in a slab, Eq. 22-23: T = g + a (g + mu), mu <- b (g + mu), mu the
// adjoint of the CPML memory), or 0 where the forward loop does not update
// the sample; g is the scaled adjoint with the term's sign (-dt/mu0
// lambda_H for the H update, dt/eps lambda_E for the E update).  T[2c+t]
// belongs to component c and its term t (0: derivative along c+1, 1: along
// c+2).  The epilogue of a gather forms T for the other half step (it is
// pointwise); the next gather applies the transposed FD rows to it.

// A quad is 4 x-adjacent samples starting on a 16-byte boundary of the
// field rows.
__device__ __forceinline__ float4 ldf4(const float *p, size_t id) { return *reinterpret_cast<const float4 *>(p + id); }
__device__ __forceinline__ void stf4(float *p, size_t id, const float4 &v) { *reinterpret_cast<float4 *>(p + id) = v; }
__device__ __forceinline__ float4 scl4(float c, const float4 &v) { return make_float4(c * v.x, c * v.y, c * v.z, c * v.w); }
// is every sample of the quad outside the CPML slabs and updated (lo .. hi
// per axis)?
__device__ __forceinline__ bool quad_plain(const AdjParams &a, const int *idx, int lo, const int *hi) {
  return idx[0] >= lo && idx[0] + 3 <= hi[0] && idx[1] >= lo && idx[1] <= hi[1] && idx[2] >= lo && idx[2] <= hi[2];
}

__device__ __forceinline__ float lane(const float4 &v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void set_lane(float4 &v, int e, float x) {
  if (e == 0) v.x = x;
  else if (e == 1) v.y = x;
  else if (e == 2) v.z = x;
  else v.w = x;
}

// The per-derivative adjoints of a quad that touches a CPML slab or a sample
// the forward loop leaves alone (KIND 0: the H_c samples, T from lambda_H;
// KIND 1: the E_c samples, T from dt/eps lambda_E, and the gradient term).
// Every array moves as float4: the CPML memory adjoints use the forward
// kernels' layouts, where a quad's four slab entries along y or z share a
// row, and along x sit at the quad's storage column (no two quads share a
// float4); lanes outside the slab or the update region keep their memory
// adjoint and get T = 0 where the forward loop does not update them.
template <int KIND>
__device__ void pre_quad(const AdjParams &a, const int *idx, const float4 (&lam4)[3]) {
  const int R = a.rd, nb = a.nb, i0 = idx[0], j = idx[1], k = idx[2];
  const size_t id = fid(a, i0, j, k);
  const int lo = KIND == 0 ? R - 1 : R;  // first sample with every FD row
  bool inx[4], rx[4];
  int sxl[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int ii = i0 + e;
    inx[e] = ii >= 0 && ii < a.np[0];
    rx[e] = ii >= lo && ii <= a.np[0] - 1 - R;
    sxl[e] = KIND == 0 ? slab_half(ii, a.np[0], nb) : slab_int(ii, a.np[0], nb);
  }
  const bool ry = j >= lo && j <= a.np[1] - 1 - R, rz = k >= lo && k <= a.np[2] - 1 - R;
  const int sy = KIND == 0 ? slab_half(j, a.np[1], nb) : slab_int(j, a.np[1], nb);
  const int sz = KIND == 0 ? slab_half(k, a.np[2], nb) : slab_int(k, a.np[2], nb);
  // storage column of the quad in the x-derivative memory arrays
  const int last = KIND == 0 ? a.np[0] - 2 : a.np[0] - 1, h = KIND == 0 ? 1 : 0;
  const int xs = i0 < nb ? i0 : ((i0 + 3 >= a.psx_far0[h] && i0 <= last) ? a.psx_hx[h] + (i0 - a.psx_far0[h]) : -1);
  const float *pml_a[3], *pml_b[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    pml_a[ax] = a.pml[ax] + (KIND == 0 ? 4 * nb : 0);
    pml_b[ax] = pml_a[ax] + 2 * nb;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int p = (c + 1) % 3, q = (c + 2) % 3;
    float4 g;
    if (KIND == 0) {
      g = scl4(-a.kappa, lam4[c]);
    } else {
      const float4 lam = lam4[c], ie = ldf4(a.ie[c], id), e0 = ldf4(a.E0[c], id), e1 = ldf4(a.E1[c], id);
      float4 gs = ldf4(a.gseg[c], id);
      const float cg = a.inv_2w0dt;
      gs.x -= lam.x * (e1.x - e0.x) * ie.x * cg;
      gs.y -= lam.y * (e1.y - e0.y) * ie.y * cg;
      gs.z -= lam.z * (e1.z - e0.z) * ie.z * cg;
      gs.w -= lam.w * (e1.w - e0.w) * ie.w * cg;
      stf4(a.gseg[c], id, gs);
      g = make_float4(ie.x * lam.x, ie.y * lam.y, ie.z * lam.z, ie.w * lam.w);
    }
#pragma unroll
    for (int term = 0; term < 2; ++term) {
      const int ax = term == 0 ? p : q;
      float4 t = term == 0 ? g : scl4(-1.f, g);
      bool on[4], any = false;
      int sl[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        bool valid = inx[e] && (p == 0 ? rx[e] : (p == 1 ? ry : rz)) && (q == 0 ? rx[e] : (q == 1 ? ry : rz));
        if (KIND == 1) valid = valid && (c == 0 ? i0 + e <= a.np[0] - 2 : (c == 1 ? j <= a.np[1] - 2 : k <= a.np[2] - 2));
        if (!valid) set_lane(t, e, 0.f);
        sl[e] = ax == 0 ? sxl[e] : (ax == 1 ? sy : sz);
        on[e] = valid && sl[e] >= 0;
        any = any || on[e];
      }
      if (any) {
        float *mu = KIND == 0 ? a.muH[2 * c + term] : a.muE[2 * c + term];
        const size_t mi = ax == 1 ? (static_cast<size_t>(k) * (2 * nb) + sy) * a.pitch + i0
                          : ax == 2 ? (static_cast<size_t>(sz) * a.np[1] + j) * a.pitch + i0
                                    : (static_cast<size_t>(k) * a.np[1] + j) * a.psx_wx[h] + xs;
        float4 m4 = ldf4(mu, mi);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (!on[e]) continue;
          const float te = lane(t, e), gp = te + lane(m4, e);
          set_lane(m4, e, pml_b[ax][sl[e]] * gp);
          set_lane(t, e, fmaf(pml_a[ax][sl[e]], gp, te));
        }
        stf4(mu, mi, m4);
      }
      stf4(KIND == 0 ? a.TH[2 * c + term] : a.TE[2 * c + term], id, t);
    }
  }
}

// The per-derivative adjoints of one quad from its final lambda values:
// KIND 0, T_H at the H_c samples from lambda_H (for the H update of the
// step before); KIND 1, the gradient term of this step, g_seg_e -=
// lambda_E_e (E1_e - E0_e) ie_e / (2 omega0 dt), and T_E at the E_e samples
// from lambda_E.  Quads inside the CPML-free region where every sample is
// updated take a float4 path without masks; the others pre_quad.
template <int KIND>
__device__ __forceinline__ void quad_terms(const AdjParams &a, const int *idx, const float4 (&lam)[3]) {
  // CPML-free samples with every FD row: nb .. np-2-nb (H) or nb .. np-1-nb (E)
  const int d = KIND == 0 ? 2 : 1;
  const int hi[3] = {a.np[0] - d - a.nb, a.np[1] - d - a.nb, a.np[2] - d - a.nb};
  if (!quad_plain(a, idx, a.nb, hi)) {
    pre_quad<KIND>(a, idx, lam);
    return;
  }
  const size_t id = fid(a, idx[0], idx[1], idx[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float4 g;
    if (KIND == 0) {
      g = scl4(-a.kappa, lam[c]);
    } else {
      const float4 ie = ldf4(a.ie[c], id), e0 = ldf4(a.E0[c], id), e1 = ldf4(a.E1[c], id);
      float4 gs = ldf4(a.gseg[c], id);
      const float cg = a.inv_2w0dt;
      gs.x -= lam[c].x * (e1.x - e0.x) * ie.x * cg;
      gs.y -= lam[c].y * (e1.y - e0.y) * ie.y * cg;
      gs.z -= lam[c].z * (e1.z - e0.z) * ie.z * cg;
      gs.w -= lam[c].w * (e1.w - e0.w) * ie.w * cg;
      stf4(a.gseg[c], id, gs);
      g = make_float4(ie.x * lam[c].x, ie.y * lam[c].y, ie.z * lam[c].z, ie.w * lam[c].w);
    }
    float *const *T = KIND == 0 ? a.TH : a.TE;
    stf4(T[2 * c], id, g);
    stf4(T[2 * c + 1], id, scl4(-1.f, g));
  }
}

// 2. Receivers at step n: lambda_c[stencil] += w * Re(sum_f cw f_n).
__global__ void k_adj_receivers(const AdjParams a, int n) {
  wait_prior_grid();
  allow_next_launch();
  const int M = 2 * a.rd, M3 = M * M * M;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nrec * 6 * M3) return;
  const int node = t % M3, rc = t / M3, c = rc % 6;
  const double *fac = (c < 3 ? a.fE : a.fH) + static_cast<size_t>(n) * a.nf * 2;
  double g = 0.0;
  for (int f = 0; f < a.nf; ++f) {
    const double *w = a.cw + (static_cast<size_t>(rc) * a.nf + f) * 2;
    g += w[0] * fac[2 * f] - w[1] * fac[2 * f + 1];
  }
  const int q1 = node % M, q2 = (node / M) % M, q3 = node / (M * M);
  const int *st = a.rec_start + rc * 3;
  const double *wt = a.rec_w + static_cast<size_t>(rc) * 3 * M;
  const double val = wt[q1] * wt[M + q2] * wt[2 * M + q3] * g;
  float *F = c < 3 ? a.lamE[c] : a.lamH[c - 3];
  atomicAdd(F + fid(a, st[0] + q1, st[1] + q2, st[2] + q3), static_cast<float>(val));
}

// ---- 1b / 4. The transposed FD gathers, TMA-fed --------------------------
// out_o += (D_{o+2})^T T[2(o+1)+0] + (D_{o+1})^T T[2(o+2)+1], with the
// transposed D+ rows into lambda_E (KIND 0, taps -R .. R-1) or the transposed
// D- rows into lambda_H (KIND 1, taps -R+1 .. R).  A CTA owns 32 x 8 columns x
// GZ planes, one thread per quad of 4 x-adjacent cells; each T array arrives
// by one bulk tensor copy with a halo along the one axis its term
// differentiates.  Every T value already holds the CPML and the update
// masks, so every CTA takes the same path.
constexpr int GX = 32, GY = 8, GZ = 2, GH = 4, GT = (GX / 4) * GY * GZ;
template <int R>
struct GTiles {
  static constexpr int YB = GX * (GY + 2 * R) * GZ;   // y-halo box: T[0], T[5]
  static constexpr int ZB = GX * GY * (GZ + 2 * R);   // z-halo box: T[1], T[2]
  static constexpr int XB = (GX + 2 * GH) * GY * GZ;  // x-halo box: T[3], T[4]
  __host__ __device__ static constexpr int off(int t) {
    return t == 0 ? 0 : t == 5 ? YB : t == 1 ? 2 * YB : t == 2 ? 2 * YB + ZB : t == 3 ? 2 * YB + 2 * ZB
                                                                                       : 2 * YB + 2 * ZB + XB;
  }
  static constexpr int FLOATS = 2 * (YB + ZB + XB);
};
struct GMaps {
  CUtensorMap m[6];
};

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int R, int KIND>
__global__ void __launch_bounds__(GT) k_adj_gather(const AdjParams a, const __grid_constant__ GMaps tm) {
  wait_prior_grid();
  allow_next_launch();
  using G = GTiles<R>;
  constexpr int M = 2 * R, OFF = KIND == 0 ? -R : 1 - R;
  extern __shared__ unsigned char smem_raw[];
  float *s = reinterpret_cast<float *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  uint64_t *bar = reinterpret_cast<uint64_t *>(s + G::FLOATS);
  // the lambda_H gather walks the tiles in the reverse of the lambda_E
  // gather's order (CTAs are dispatched in index order), so each gather
  // starts on the tiles whose inputs the one before touched last (in L2)
  const int bx = KIND == 0 ? static_cast<int>(blockIdx.x) : static_cast<int>(gridDim.x - 1 - blockIdx.x);
  const int by = KIND == 0 ? static_cast<int>(blockIdx.y) : static_cast<int>(gridDim.y - 1 - blockIdx.y);
  const int bz = KIND == 0 ? static_cast<int>(blockIdx.z) : static_cast<int>(gridDim.z - 1 - blockIdx.z);
  const int i0 = a.org[0] + bx * GX, j0 = a.org[1] + by * GY, k0 = bz * GZ;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    mbar_expect_tx(bar, static_cast<uint32_t>(G::FLOATS * 4));
    tma_load_3d(s + G::off(0), &tm.m[0], bar, i0, j0 - R, k0);
    tma_load_3d(s + G::off(5), &tm.m[5], bar, i0, j0 - R, k0);
    tma_load_3d(s + G::off(1), &tm.m[1], bar, i0, j0, k0 - R);
    tma_load_3d(s + G::off(2), &tm.m[2], bar, i0, j0, k0 - R);
    tma_load_3d(s + G::off(3), &tm.m[3], bar, i0 - GH, j0, k0);
    tma_load_3d(s + G::off(4), &tm.m[4], bar, i0 - GH, j0, k0);
  }
  const int t = threadIdx.x, q4 = 4 * (t & 7), r = (t >> 3) & 7, c = t >> 6;
  const int i = i0 + q4, j = j0 + r, k = k0 + c;
  const bool live = i >= 0 && i < a.np[0] && j < a.np[1] && k < a.np[2];
  float *const *out = KIND == 0 ? a.lamE : a.lamH;
  const float *const *tab = KIND == 0 ? a.cpT : a.cmT;
  const size_t id = fid(a, live ? i : 0, live ? j : 0, live ? k : 0);
  float4 o4[3];
#pragma unroll
  for (int o = 0; o < 3; ++o) o4[o] = live ? *reinterpret_cast<const float4 *>(out[o] + id) : float4{};
  if (KIND == 0 && live) {
    // the epilogue's inputs (dt/eps, the E snapshots, the gradient term),
    // brought into L2 while the tiles are in flight
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      prefetch_l2(a.ie[c] + id);
      prefetch_l2(a.E0[c] + id);
      prefetch_l2(a.E1[c] + id);
      prefetch_l2(a.gseg[c] + id);
    }
  }
  float cx[4][M], cy[M], cz[M];
#pragma unroll
  for (int f = 0; f < M; ++f) {
    const float4 v = live ? __ldg(reinterpret_cast<const float4 *>(tab[0] + static_cast<size_t>(i) * M) + f) : float4{};
    cx[(4 * f) / M][(4 * f) % M] = v.x;
    cx[(4 * f + 1) / M][(4 * f + 1) % M] = v.y;
    cx[(4 * f + 2) / M][(4 * f + 2) % M] = v.z;
    cx[(4 * f + 3) / M][(4 * f + 3) % M] = v.w;
    cy[f] = live ? __ldg(tab[1] + static_cast<size_t>(j) * M + f) : 0.f;
    cz[f] = live ? __ldg(tab[2] + static_cast<size_t>(k) * M + f) : 0.f;
  }
  __syncthreads();
  int late = 0;
  if (threadIdx.x == 0 && !mbar_wait_bounded(bar, 0)) {
    late = 1;
    atomicExch(a.status, EMM_ETIMEOUT);
    mbar_wait_bounded(bar, 0);
  }
  if (__syncthreads_or(late) || !live) return;

  // taps of term array tt along axis ax for the quad, accumulated into acc
  auto ybox = [&](int tt, int row) {
    return *reinterpret_cast<const float4 *>(s + G::off(tt) + (c * (GY + 2 * R) + row) * GX + q4);
  };
  auto zbox = [&](int tt, int plane) {
    return *reinterpret_cast<const float4 *>(s + G::off(tt) + (plane * GY + r) * GX + q4);
  };
  auto xrow = [&](int tt, float *row) {
    const float *b = s + G::off(tt) + (c * GY + r) * (GX + 2 * GH) + q4;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const float4 v = *reinterpret_cast<const float4 *>(b + 4 * u);
      row[4 * u] = v.x; row[4 * u + 1] = v.y; row[4 * u + 2] = v.z; row[4 * u + 3] = v.w;
    }
  };
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const int ta = 2 * ((o + 1) % 3), aa = (o + 2) % 3, tb = 2 * ((o + 2) % 3) + 1, ab = (o + 1) % 3;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int term = 0; term < 2; ++term) {
      const int tt = term == 0 ? ta : tb, ax = term == 0 ? aa : ab;
      if (ax == 0) {
        float row[12];
        xrow(tt, row);
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int m = 0; m < M; ++m) acc[e] = fmaf(cx[e][m], row[GH + e + OFF + m], acc[e]);
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float4 v = ax == 1 ? ybox(tt, r + R + OFF + m) : zbox(tt, c + R + OFF + m);
          const float cf = ax == 1 ? cy[m] : cz[m];
          acc[0] = fmaf(cf, v.x, acc[0]);
          acc[1] = fmaf(cf, v.y, acc[1]);
          acc[2] = fmaf(cf, v.z, acc[2]);
          acc[3] = fmaf(cf, v.w, acc[3]);
        }
      }
    }
    if (i + 0 < a.np[0]) o4[o].x += acc[0];
    if (i + 1 < a.np[0]) o4[o].y += acc[1];
    if (i + 2 < a.np[0]) o4[o].z += acc[2];
    if (i + 3 < a.np[0]) o4[o].w += acc[3];
    *reinterpret_cast<float4 *>(out[o] + id) = o4[o];
  }
  // epilogue: the pointwise terms that read the lambda just completed
  // (lambda_E of this step after the receivers, or lambda_H for the step
  // before), owned by this quad
  const int idx[3] = {i, j, k};
  quad_terms<KIND == 0 ? 1 : 0>(a, idx, o4);
}

// E snapshots: a streaming copy of the three E arrays (float4), launched as a
// programmatic dependent like the steps around it.
__global__ void k_copy16(const float4 *src, float4 *dst, size_t n) {
  wait_prior_grid();
  allow_next_launch();
  for (size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[t] = src[t];
}

// End of a checkpoint segment: g_pad += g_seg (FP64), g_seg = 0.
__global__ void k_adj_flush(const AdjParams a) {
  int idx[3];
  if (!cell3(a, idx)) return;
  const size_t id = fid(a, idx[0], idx[1], idx[2]);
  for (int c = 0; c < 3; ++c) {
    const float g = a.gseg[c][id];
    if (g != 0.f) {
      a.gpad[c][id] += static_cast<double>(g);
      a.gseg[c][id] = 0.f;
    }
  }
}

// cw[r][c][f] = conj(v) * norm[c < 3 ? 0 : 1][f]  (Eq. 7 normalisation).
// Least-squares residual of the forward sweep's Green's functions: r =
// w (G - d) (the cotangent of the misfit 1/2 sum w |G - d|^2, which is added
// to *misfit).  One block; the tree reduction fixes the summation order.
constexpr int kResThreads = 256;
__global__ void __launch_bounds__(kResThreads)
    k_residual(const double *G, const double *d, const double *wt, double *r, double *misfit, int n) {
  __shared__ double part[kResThreads];
  double acc = 0.0;
  for (int t = threadIdx.x; t < n; t += kResThreads) {
    const double re = G[2 * t] - d[2 * t], im = G[2 * t + 1] - d[2 * t + 1], w = wt ? wt[t] : 1.0;
    r[2 * t] = w * re;
    r[2 * t + 1] = w * im;
    acc += 0.5 * w * (re * re + im * im);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kResThreads / 2; h > 0; h /= 2) {
    if (static_cast<int>(threadIdx.x) < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *misfit += part[0];
}

__global__ void k_adj_weights(const double *v, const double *norm, double *cw, int nrec, int nf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrec * 6 * nf) return;
  const int f = t % nf, c = (t / nf) % 6;
  const double vr = v[2 * t], vi = -v[2 * t + 1];
  const double *nm = norm + ((c < 3 ? 0 : 1) * nf + f) * 2;
  cw[2 * t] = vr * nm[0] - vi * nm[1];
  cw[2 * t + 1] = vr * nm[1] + vi * nm[0];
}

// Fold the padded gradient onto the interior samples: every padded sample
// holds the value of the interior sample its clamped index names.
__global__ void k_adj_fold(const AdjParams a, double *grad) {
  const size_t nint = static_cast<size_t>(a.n[0]) * a.n[1] * a.n[2];
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < 3 * nint;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(t / nint);
    const size_t r = t % nint;
    const int ii = static_cast<int>(r % a.n[0]), jj = static_cast<int>((r / a.n[0]) % a.n[1]),
              kk = static_cast<int>(r / (static_cast<size_t>(a.n[0]) * a.n[1]));
    int lo[3], hi[3];
    const int in[3] = {ii, jj, kk};
    for (int ax = 0; ax < 3; ++ax) {
      lo[ax] = in[ax] == 0 ? 0 : in[ax] + a.nbe;
      hi[ax] = in[ax] == a.n[ax] - 1 ? a.np[ax] - 1 : in[ax] + a.nbe;
    }
    double s = 0.0;
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) s += a.gpad[c][fid(a, i, j, k)];
    grad[t] = s;
  }
}

// 3-D FP32 tensor [np2][np1][pitch] (dims np0 x np1 x np2), box bx x by x bz.
bool make_map3(CUtensorMap *map, const float *base, const AdjParams &a, int bx, int by, int bz) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(a.np[0]), static_cast<cuuint64_t>(a.np[1]),
                              static_cast<cuuint64_t>(a.np[2])};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(a.pitch) * 4, static_cast<cuuint64_t>(a.plane) * 4};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(bx), static_cast<cuuint32_t>(by), static_cast<cuuint32_t>(bz)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The two gathers of one adjoint step, for order R.
struct Gathers {
  GMaps maps0, maps1;  // T_H for the lambda_E gather, T_E for the lambda_H gather
  dim3 grid;
  size_t smem;
  void (*g0)(AdjParams, GMaps);
  void (*g1)(AdjParams, GMaps);
};
template <int R>
bool make_gathers(const AdjParams &a, Gathers *G) {
  bool ok = true;
  for (int t = 0; t < 6 && ok; ++t) {
    const int bx = (t == 3 || t == 4) ? GX + 2 * GH : GX;
    const int by = (t == 0 || t == 5) ? GY + 2 * R : GY;
    const int bz = (t == 1 || t == 2) ? GZ + 2 * R : GZ;
    ok = make_map3(&G->maps0.m[t], a.TH[t], a, bx, by, bz) && make_map3(&G->maps1.m[t], a.TE[t], a, bx, by, bz);
  }
  G->grid = dim3((a.np[0] - a.org[0] + GX - 1) / GX, (a.np[1] - a.org[1] + GY - 1) / GY, (a.np[2] + GZ - 1) / GZ);
  G->smem = GTiles<R>::FLOATS * 4 + 128 + 16;
  G->g0 = k_adj_gather<R, 0>;
  G->g1 = k_adj_gather<R, 1>;
  ok = ok && cudaFuncSetAttribute(k_adj_gather<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(G->smem)) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_adj_gather<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(G->smem)) == cudaSuccess;
  return ok;
}

// Byte layout of the gradient's extra workspace, after the forward one.
struct AdjLayout {
  size_t fwd, ck, state, nck, eh, ebytes, first_stored, snap, lamE[3], lamH[3], TH[6], TE[6], muE[6], muH[6], gpad[3], gseg[3], cpT[3], cmT[3], cw,
      res, total;
};

// K: steps between checkpoints; S: a budget of steps whose E snapshots the
// forward sweep keeps (whole checkpoint segments from the end of the run),
// so that the reverse sweep need not recompute them.
AdjLayout adj_plan(const emm_grid *g, const emm_survey *s, int K, int S) {
  AdjLayout A{};
  const Layout L = plan(g, s);
  const FieldGeom fg = field_geom(g);
  size_t off = L.total;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t cells = static_cast<size_t>(fg.pitch) * g->ax[1].npad * g->ax[2].npad;
  const int nt = s->nt > 0 ? s->nt : 0;
  A.fwd = L.total;
  A.state = L.sstride;                     // E, H and the CPML memory
  A.ebytes = L.H[0] - L.E[0];              // E only
  A.nck = nt > 0 ? static_cast<size_t>((nt + K - 1) / K) : 0;
  // segments first_stored .. nck-1 keep E^{first_stored K} .. E^{nt} from the forward sweep
  const size_t ns = std::min<size_t>(A.nck, static_cast<size_t>(S > 0 ? S : 0) / static_cast<size_t>(K));
  A.first_stored = A.nck - ns;
  A.ck = take(A.first_stored * A.state);
  A.eh = take(A.first_stored > 0 ? static_cast<size_t>(K) * A.ebytes : 0);  // E^{it0+1} .. E^{it0+K}
  A.snap = take(ns > 0 ? (static_cast<size_t>(nt) - A.first_stored * K + 1) * A.ebytes : 0);
  for (int c = 0; c < 3; ++c) A.lamE[c] = take(cells * 4);
  for (int c = 0; c < 3; ++c) A.lamH[c] = take(cells * 4);
  for (int c = 0; c < 6; ++c) A.TH[c] = take(cells * 4);
  for (int c = 0; c < 6; ++c) A.TE[c] = take(cells * 4);
  for (int c = 0; c < 6; ++c) A.muE[c] = take((c < 5 ? L.psiE[c + 1] : L.psiH[0]) - L.psiE[c]);
  for (int c = 0; c < 6; ++c) A.muH[c] = take((c < 5 ? L.psiH[c + 1] : L.E[0] + L.sstride) - L.psiH[c]);
  for (int c = 0; c < 3; ++c) A.gpad[c] = take(cells * 8);
  for (int c = 0; c < 3; ++c) A.gseg[c] = take(cells * 4);
  const size_t m = 2 * static_cast<size_t>(g->rd);
  // the x tables run on to a whole field row (zero rows past npad): the
  // gathers read the rows of all four cells of a quad at once
  const size_t xrows = std::max<size_t>(g->ax[0].npad, fg.pitch);
  for (int a = 0; a < 3; ++a) A.cpT[a] = take((a == 0 ? xrows : g->ax[a].npad) * m * 4);
  for (int a = 0; a < 3; ++a) A.cmT[a] = take((a == 0 ? xrows : g->ax[a].npad) * m * 4);
  A.cw = take(static_cast<size_t>(s->nrec > 0 ? s->nrec : 1) * 6 * s->nfreq * 2 * sizeof(double));
  A.res = take(static_cast<size_t>(s->nrec > 0 ? s->nrec : 1) * 6 * s->nfreq * 2 * sizeof(double));
  A.total = off;
  return A;
}

// Transposed FD rows in gather form.  D+ row r (half sample r, valid for
// rd-1 <= r <= npad-1-rd) reads integer samples r-rd+1 .. r+rd; its transpose
// at integer sample i gathers rows r = i-rd+q, q = 0..2rd-1, with coefficient
// cp[r][2rd-1-q].  D- row r (integer sample, valid rd <= r <= npad-1-rd)
// reads half samples r-rd .. r+rd-1; its transpose at half sample i gathers
// rows r = i-rd+1+q with coefficient cm[r][2rd-1-q].  Invalid rows give 0.
void transposed_rows(const Axis &ax, int rd, std::vector<float> &pT, std::vector<float> &mT) {
  const int np = ax.npad, M = 2 * rd;
  pT.assign(static_cast<size_t>(np) * M, 0.f);
  mT.assign(static_cast<size_t>(np) * M, 0.f);
  for (int i = 0; i < np; ++i)
    for (int q = 0; q < M; ++q) {
      const int rp = i - rd + q;
      if (rp >= rd - 1 && rp <= np - 1 - rd) pT[static_cast<size_t>(i) * M + q] = static_cast<float>(ax.cp[static_cast<size_t>(rp) * M + M - 1 - q]);
      const int rm = i - rd + 1 + q;
      if (rm >= rd && rm <= np - 1 - rd) mT[static_cast<size_t>(i) * M + q] = static_cast<float>(ax.cm[static_cast<size_t>(rm) * M + M - 1 - q]);
    }
}

// With d_obs set, the cotangent is the misfit residual w (G - d_obs) of the
// forward sweep's own G (dG unused), and the misfit is added to *misfit.
int gradient_impl(const emm_grid *g, const emm_survey *s, const float *sigma, const double *dG, int K, int S,
                  void *ws, size_t ws_bytes, double *rec_out, double *grad, cudaStream_t cs,
                  const double *d_obs = nullptr, const double *wts = nullptr, double *misfit = nullptr) {
  int st = check_survey(g, s);
  if (st != EMM_OK) return st;
  if (K < 1 || s->volume || s->src_kind != 0 || s->src_length > 0 || s->airwave || !grad || !sigma || !ws ||
      (s->nrec > 0 && ((!dG && !d_obs) || !rec_out)) || (d_obs && !misfit))
    return EMM_EINVAL;
  if (S < 0) return EMM_EINVAL;
  const AdjLayout A = adj_plan(g, s, K, S);
  if (ws_bytes < A.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return EMM_EWORKSPACE;
  Prepared P;
  st = prepare_forward(g, s, sigma, ws, A.fwd, rec_out, nullptr, cs, &P, 1, nullptr, false, true, 0);
  if (st != EMM_OK) return st;
  unsigned char *base = static_cast<unsigned char *>(ws);
  const Layout &L = P.L;
  const int nt = s->nt, nf = s->nfreq, rd = g->rd;

  // forward sweep with checkpoints, then, over the stored segments, every
  // E snapshot; the receivers accumulate G on the way
  cudaError_t e = cudaSuccess;
  const int base_step = static_cast<int>(A.first_stored) * K;
  auto snap = [&](int n) { return base + A.snap + static_cast<size_t>(n - base_step) * A.ebytes; };
  // the E arrays (A.ebytes, a multiple of 256) from the state into a snapshot
  const dim3 cgrid(static_cast<unsigned>(4 * P.sms));
  auto copy_e = [&](unsigned char *dst) {
    return launch_dependent(k_copy16, cgrid, dim3(256), 0, cs, reinterpret_cast<const float4 *>(base + L.E[0]),
                            reinterpret_cast<float4 *>(dst), A.ebytes / 16);
  };
  // one step from the E arrays at src to those at dst (snapshot-shaped
  // blocks, src == nullptr for the state's own arrays): the E half-step
  // writes E^{n+1} there and the rest of the step reads it there
  auto step_into = [&](const DevParams &p0, dim3 blocks, int it, unsigned char *src, unsigned char *dst) {
    DevParams q = p0;
    for (int c = 0; c < 3; ++c) {
      const size_t ec = L.E[c] - L.E[0];
      if (src) q.E[c] = reinterpret_cast<float *>(src + ec) + P.fg.xshift;
      q.Eout[c] = reinterpret_cast<float *>(dst + ec) + P.fg.xshift;
    }
    return run_steps(P, q, blocks, it, it + 1, cs, nullptr);
  };
  for (int it0 = 0; it0 < nt && e == cudaSuccess; it0 += K) {
    const int it1 = std::min(it0 + K, nt);
    if (it0 < base_step) {
      e = cudaMemcpyAsync(base + A.ck + static_cast<size_t>(it0 / K) * A.state, base + L.E[0], A.state,
                          cudaMemcpyDeviceToDevice, cs);
      if (e == cudaSuccess) e = run_steps(P, P.p, P.blocks, it0, it1, cs, nullptr);
      continue;
    }
    if (it0 == base_step) e = copy_e(snap(it0));
    for (int it = it0; it < it1 && e == cudaSuccess; ++it) e = step_into(P.p, P.blocks, it, snap(it), snap(it + 1));
  }
  if (e != cudaSuccess) return EMM_ECUDA;
  st = finalize_forward(P, s, rec_out, nullptr, cs);
  if (st != EMM_OK) return st;

  // adjoint state and tables
  AdjParams a{};
  for (int ax = 0; ax < 3; ++ax) {
    a.np[ax] = P.p.np[ax];
    a.n[ax] = P.p.n[ax];
    a.pml[ax] = P.p.pml[ax];
    a.cpT[ax] = reinterpret_cast<const float *>(base + A.cpT[ax]);
    a.cmT[ax] = reinterpret_cast<const float *>(base + A.cmT[ax]);
  }
  a.pitch = P.p.pitch;
  a.plane = P.p.plane;
  a.nb = g->nb;
  a.rd = rd;
  a.nbe = P.p.nbe;
  for (int ax = 0; ax < 3; ++ax) a.org[ax] = P.p.org[ax];
  a.status = P.p.status;
  a.kappa = P.p.dt_mu;
  a.inv_2w0dt = static_cast<float>(1.0 / (2.0 * s->omega0 * P.dt));
  const int xs = P.fg.xshift;
  for (int c = 0; c < 3; ++c) {
    a.ie[c] = P.p.ie[c];
    a.lamE[c] = reinterpret_cast<float *>(base + A.lamE[c]) + xs;
    a.lamH[c] = reinterpret_cast<float *>(base + A.lamH[c]) + xs;
    a.gpad[c] = reinterpret_cast<double *>(base + A.gpad[c]) + xs;
    a.gseg[c] = reinterpret_cast<float *>(base + A.gseg[c]) + xs;
  }
  for (int c = 0; c < 6; ++c) {
    a.TH[c] = reinterpret_cast<float *>(base + A.TH[c]) + xs;
    a.TE[c] = reinterpret_cast<float *>(base + A.TE[c]) + xs;
    const int shift = psi_axis(c) == 0 ? 0 : xs;
    a.muE[c] = reinterpret_cast<float *>(base + A.muE[c]) + shift;
    a.muH[c] = reinterpret_cast<float *>(base + A.muH[c]) + shift;
  }
  for (int h = 0; h < 2; ++h) {
    a.psx_hx[h] = P.p.psx_hx[h];
    a.psx_wx[h] = P.p.psx_wx[h];
    a.psx_far0[h] = P.p.psx_far0[h];
  }
  a.nrec = s->nrec;
  a.nf = nf;
  a.rec_start = P.p.rec_start;
  a.rec_w = P.p.rec_w;
  a.cw = reinterpret_cast<const double *>(base + A.cw);
  a.fE = P.p.fE;
  a.fH = P.p.fH;

  // everything from the first adjoint field to the gradient starts at zero
  e = cudaMemsetAsync(base + A.lamE[0], 0, A.cpT[0] - A.lamE[0], cs);
  std::vector<float> pT, mT;
  for (int ax = 0; ax < 3 && e == cudaSuccess; ++ax) {
    transposed_rows(g->ax[ax], rd, pT, mT);
    if (ax == 0) {
      const size_t rows = std::max<size_t>(g->ax[0].npad, P.fg.pitch) * 2 * rd;
      pT.resize(rows, 0.f);
      mT.resize(rows, 0.f);
    }
    e = cudaMemcpyAsync(base + A.cpT[ax], pT.data(), pT.size() * 4, cudaMemcpyHostToDevice, cs);
    // pageable sources: each copy has taken the data when it returns
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + A.cmT[ax], mT.data(), mT.size() * 4, cudaMemcpyHostToDevice, cs);
  }
  if (e != cudaSuccess) return EMM_ECUDA;
  if (s->nrec > 0) {
    const int tot = s->nrec * 6 * nf;
    if (d_obs) {
      double *res = reinterpret_cast<double *>(base + A.res);
      k_residual<<<1, kResThreads, 0, cs>>>(rec_out, d_obs, wts, res, misfit, tot);
      dG = res;
    }
    k_adj_weights<<<(tot + 255) / 256, 256, 0, cs>>>(dG, reinterpret_cast<const double *>(base + L.norm),
                                                     reinterpret_cast<double *>(base + A.cw), s->nrec, nf);
  }

  // recomputation runs without receivers (G is already accumulated)
  DevParams pr = P.p;
  pr.nrec = 0;
  pr.rec_blocks = 0;
  pr.rec_layers = 0;
  const dim3 blocks_r(P.p.tiles_x, P.p.tiles_y, P.p.tiles_z);
  const int grid_cells = P.sms * 8;
  const dim3 tb(32, 8, 1), grid3((P.p.np[0] + 31) / 32, (P.p.np[1] + 7) / 8, P.p.np[2]);
  // pre passes: 32 x 4 threads, 4 x-adjacent samples each, over x from org[0]
  Gathers GA{};
  const bool gok = rd == 1 ? make_gathers<1>(a, &GA)
                   : rd == 2 ? make_gathers<2>(a, &GA)
                             : rd == 3 ? make_gathers<3>(a, &GA) : make_gathers<4>(a, &GA);
  if (!gok) return EMM_ECUDA;

  const int M = 2 * rd, rec_threads = s->nrec * 6 * M * M * M;
  for (int seg = static_cast<int>(A.nck) - 1; seg >= 0 && e == cudaSuccess; --seg) {
    const int it0 = seg * K, it1 = std::min(it0 + K, nt);
    const bool stored = static_cast<size_t>(seg) >= A.first_stored;
    // E snapshot of step n: kept by the forward sweep, or recomputed here
    // from the checkpoint (whose leading bytes are the E arrays of step it0)
    unsigned char *ck = base + A.ck + static_cast<size_t>(seg) * A.state;
    auto esnap = [&](int n) {
      return stored ? snap(n) : n == it0 ? ck : base + A.eh + static_cast<size_t>(n - it0 - 1) * A.ebytes;
    };
    if (!stored) {
      e = cudaMemcpyAsync(base + L.E[0], ck, A.state, cudaMemcpyDeviceToDevice, cs);
      for (int it = it0; it < it1 && e == cudaSuccess; ++it) e = step_into(pr, blocks_r, it, esnap(it), esnap(it + 1));
    }
    for (int it = it1 - 1; it >= it0 && e == cudaSuccess; --it) {
      for (int c = 0; c < 3; ++c) {
        const size_t ec = L.E[c] - L.E[0];
        a.E0[c] = reinterpret_cast<const float *>(esnap(it) + ec) + xs;
        a.E1[c] = reinterpret_cast<const float *>(esnap(it + 1) + ec) + xs;
      }
      // T_H of this step came from the lambda_H gather of the step after it
      // (zero for the last step); the receivers add to lambda before the
      // lambda_E gather, whose epilogue forms T_E and the gradient term; the
      // lambda_H gather's epilogue forms T_H of the step before
      if (rec_threads > 0)
        e = launch_dependent(k_adj_receivers, dim3((rec_threads + kThreads - 1) / kThreads), dim3(kThreads), 0, cs,
                             a, it);
      if (e == cudaSuccess) e = launch_dependent(GA.g0, GA.grid, dim3(GT), GA.smem, cs, a, GA.maps0);
      if (e == cudaSuccess) e = launch_dependent(GA.g1, GA.grid, dim3(GT), GA.smem, cs, a, GA.maps1);
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_adj_flush<<<grid3, tb, 0, cs>>>(a);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return EMM_ECUDA;
  k_adj_fold<<<grid_cells, kThreads, 0, cs>>>(a, grad);
  return cudaGetLastError() == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

}  // namespace
}  // namespace emm

extern "C" {

int emm_gradient_stored_workspace_size(const emm_grid *g, const emm_survey *s, int ckpt_every, int stored_steps,
                                       size_t *bytes) {
  const int st = emm::check_survey(g, s);
  if (st != EMM_OK) return st;
  if (!bytes || ckpt_every < 1 || stored_steps < 0 || s->volume) return EMM_EINVAL;
  *bytes = emm::adj_plan(g, s, ckpt_every, stored_steps).total;
  return EMM_OK;
}

int emm_gradient_workspace_size(const emm_grid *g, const emm_survey *s, int ckpt_every, size_t *bytes) {
  return emm_gradient_stored_workspace_size(g, s, ckpt_every, 0, bytes);
}

int emm_gradient_stored(const emm_grid *g, const emm_survey *s, const float *sigma, const double *dG,
                        int ckpt_every, int stored_steps, void *ws, size_t ws_bytes, double *rec_out, double *grad,
                        emm_stream stream) {
  return emm::gradient_impl(g, s, sigma, dG, ckpt_every, stored_steps, ws, ws_bytes, rec_out, grad,
                            reinterpret_cast<cudaStream_t>(stream));
}

int emm_misfit_gradient(const emm_grid *g, const emm_survey *s, const float *sigma, const double *d_obs,
                        const double *weight, int ckpt_every, int stored_steps, void *ws, size_t ws_bytes,
                        double *rec_out, double *misfit, double *grad, emm_stream stream) {
  if (!d_obs || !misfit) return EMM_EINVAL;
  return emm::gradient_impl(g, s, sigma, nullptr, ckpt_every, stored_steps, ws, ws_bytes, rec_out, grad,
                            reinterpret_cast<cudaStream_t>(stream), d_obs, weight, misfit);
}

int emm_gradient(const emm_grid *g, const emm_survey *s, const float *sigma, const double *dG, int ckpt_every,
                 void *ws, size_t ws_bytes, double *rec_out, double *grad, emm_stream stream) {
  return emm_gradient_stored(g, s, sigma, dG, ckpt_every, 0, ws, ws_bytes, rec_out, grad, stream);
}

}  // extern "C"
