// emm_internal.h -- structures shared by the host setup (emm_setup.cpp) and
// the CUDA kernels (emm_kernels.cu) of libemm.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <vector_types.h>

#include "../../include/emm.h"

namespace emm {

constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;  // mu = mu0 everywhere
constexpr int kMaxRd = 4;

// One padded axis: nodes, half nodes, FD rows, CPML slab maps.
struct Axis {
  int n = 0, npad = 0;
  std::vector<double> X;       // npad+1 integer nodes (X[npad] bounds the last half cell)
  std::vector<double> Xh;      // npad half nodes
  std::vector<double> cp, cm;  // [npad][2rd] D+ (at Xh[i]) and D- (at X[i]) rows
  std::vector<int> cp_start;   // first tap of the D+ row (i-rd+1) or -1
  std::vector<int> cm_start;   // first tap of the D- row (i-rd) or -1
  std::vector<int> slab_i;     // CPML slab entry of integer sample i, or -1
  std::vector<int> slab_h;     // CPML slab entry of half sample i, or -1
};

}  // namespace emm

struct emm_grid {
  int rd = 0, nb = 0, ne = 0;
  emm::Axis ax[3];
};

namespace emm {

// Component staggering: 1 = half nodes along that axis.
constexpr int kHalf[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                             {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

// Host helpers implemented in emm_setup.cpp (used by emm_forward).
int locate_axis(const emm_grid *g, int axis, int half, double p, int *start, double *w);
double dmax_axis(const Axis &ax, int rd);
void cpml_axis(const emm_grid *g, int axis, double vmax, double fmax, double dt, double *ab);

// Everything the kernels read, packed by value into the launch parameters.
struct DevParams {
  int np[3];        // padded sizes
  int n[3];         // interior sizes
  int pitch;        // row pitch (samples) of the field arrays, a multiple of 32
  size_t plane;     // pitch * np[1]
  int nbe, nb;
  int org[3];       // grid coordinates of the first tile (<= 0)
  int tiles_x, tiles_y, tiles_z, stencil_blocks;  // stencil_blocks: stencil CTAs of a launch
  int rec_blocks;   // receiver CTAs (one warp per receiver component)
  int rec_layers;   // grid z layers holding them (the first ones)
  float dt_mu;      // dt / mu0
  float *E[3], *H[3];        // sample (i, j, k) at [k * plane + j * pitch + i]
  const float *ie[3];        // dt / eps = 2 omega0 dt / sigma on the padded grid
  float *psiE[6];            // CPML memory of curl H terms (E update)
  float *psiH[6];            // CPML memory of curl E terms (H update)
  int psx_hx[2], psx_wx[2], psx_far0[2];  // x-derivative CPML storage ([0] psiE, [1] psiH)
  const float *cm[3], *cp[3];  // FD rows [npad][2rd]
  const float *pml[3];         // [4][2nb]: a_int, b_int, a_half, b_half
  // source
  int src_on[3];
  int src_start[3][3];
  int src_any, src_lo[3], src_hi[3];  // bounding box of the source stencils
  const float *jw[3];          // dir_c * w / V at the (2rd)^3 stencil nodes
  const float *amp;            // [nt]: moment * wavelet(t_{n+1/2})
  // receivers
  int nrec, nf;
  const int *rec_start;        // [nrec][6][3]
  const double *rec_w;         // [nrec][6][3][2rd]
  double *rec_acc;             // [nrec][6][nf][2] (the caller's output, accumulated in place)
  const double *fE, *fH;       // [nt][nf][2] DTFT factors e^{i w' t} dt (E: t=(n+1)dt, H: (n+1/2)dt)
  // volume
  float4 *vacc;                // [6][nf][n3][n2][n1] compensated FP32 (re_hi, re_lo, im_hi, im_lo)
  const float *fE32, *fH32;    // [nt][nf][2] FP32 copies of the factors for the volume
  int *status;
};

}  // namespace emm
