// emm_internal.h -- structures shared by the host setup (emm_setup.cpp) and
// the CUDA kernels (emm_kernels.cu) of libemm.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime_api.h>
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

// Source of one transmitter of a batch: which E components it drives, the
// first node of each (2rd)^3 stencil, and their bounding box.
// Source stencil of one transmitter: per component c, weights on the box of
// samples start[c] .. start[c] + box[c] - 1 (x fastest), at float offset
// woff[c] of the transmitter's block of jw.  A point dipole has (2rd)^3
// boxes; an antenna the union of its sub-dipoles' boxes.  lo/hi: the
// bounding box of all components.
struct SrcDev {
  int on[3];
  int start[3][3];
  int any, lo[3], hi[3];
  int box[3][3], woff[3];
};

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
  // Convergence runs (else null): DTFT of the six components at the 8
  // corners of the model interior for the lowest frequency, [8][6][2] FP64,
  // followed by its value at the last check; and the stop word, nonzero once
  // the corner test has passed (every later launch then returns at once).
  double *corner;
  const int *halt;
  int conv_f;       // index of the lowest frequency
  int src_magnetic; // 1: the source is a magnetic dipole, injected in the H update
  int src_fused;    // 1: the E kernel injects J itself (an electric point dipole);
                    // otherwise k_inject does, after the E or the H launch
  size_t jstride;   // floats of jw per transmitter
  // Air above the model (airwave runs; else air_on = 0): interface row ks,
  // roots of unity e^{-2 pi i m / np} per axis ([np]), continuation factors of the E
  // rows [rd-1][np1][np0] and of the H rows [2][rd][np1][np0] (H_x, H_y),
  // and the work planes T, F [nsrc][3][np1][np0] and U [nsrc][2 rd][np1][np0].
  int air_on, air_ks, air_rd;
  const float2 *air_twx, *air_twy, *air_facH;
  const float *air_decE;
  float2 *air_T, *air_F, *air_U;
  float dt_mu;      // dt / mu0
  float *E[3], *H[3];        // sample (i, j, k) at [k * plane + j * pitch + i]
  float *Eout[3];            // set for a one-step run: the E half-step writes E^{n+1}
                             // here (same layout) and leaves E[] as it was
  float *Hout[3];            // ring runs: the H half-step writes H^{n+3/2} here
  // Field ring of a solve with the volume DTFT (ring_k > 1): slot s holds
  // E^m and H^{m+1/2} for m = s mod ring_k; slot 0 is E[] / H[] of the state,
  // slot s >= 1 component c (0..2 E, 3..5 H) starts at
  // ring + ((s - 1) * 6 + c) * ring_comp.  ring_k = 1: the fields stay in place.
  float *ring;
  size_t ring_comp;
  int ring_k;
  const float *ie[3];        // dt / eps = 2 omega0 dt / sigma on the padded grid
  float *psiE[6];            // CPML memory of curl H terms (E update)
  float *psiH[6];            // CPML memory of curl E terms (H update)
  int psx_hx[2], psx_wx[2], psx_far0[2];  // x-derivative CPML storage ([0] psiE, [1] psiH)
  const float *cm[3], *cp[3];  // FD rows [npad][2rd]
  const float *pml[3];         // [4][2nb]: a_int, b_int, a_half, b_half
  // transmitters: nsrc state blocks (fields and CPML memory) sstride floats
  // apart, sharing dt/eps, the tables and the receivers
  int nsrc;
  size_t sstride;
  const SrcDev *srcs;          // [nsrc]
  const float *jw;             // [nsrc][3][(2rd)^3]: dir_c * w / V at the stencil nodes
  const float *amp;            // [nt]: moment * wavelet(t_{n+1/2})
  // receivers
  int nrec, nf;
  const int *rec_start;        // [nrec][6][3]
  const double *rec_w;         // [nrec][6][3][2rd]
  double *rec_acc;             // [nsrc][nrec][6][nf][2] (the caller's output, accumulated in place)
  const double *fE, *fH;       // [nt][nf][2] DTFT factors e^{i w' t} dt (E: t=(n+1)dt, H: (n+1/2)dt)
  // volume
  float4 *vacc;                // [6][nf][n3][n2][n1] compensated FP32 (re_hi, re_lo, im_hi, im_lo)
  const float *fE32, *fH32;    // [nt][nf][2] FP32 copies of the factors for the volume
  int *status;
  int *abort;                  // persistent runs: set when a bounded wait ran out (else null)
};

// ---- host-side pieces shared by the forward and the gradient entry points ----
constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Tiling of the padded grid and the matching field-array geometry.  Tiles
// start at org[a] <= 0, chosen so that a tile edge falls on the first
// CPML-free sample max(nb, rd) (x: rounded down to a multiple of 4 for the
// TMA boxes), which maximises the CTAs that take the interior path.  Field
// rows hold xshift = -org[0] leading samples, so every tile row starts on a
// 128-byte line; the row pitch is a multiple of 32 samples.
struct FieldGeom {
  int org[3], tiles[3], xshift, pitch;
  int psx_hx[2], psx_wx[2], psx_far0[2];  // x-derivative CPML storage: [0] integer, [1] half samples
};
// shape: the stencil tile shape the tiling is for (0: 32 x 8 x 2, 1: 32 x 4 x 4);
// the memory layout does not depend on it.
FieldGeom field_geom(const emm_grid *g, int shape = 0);

// Byte layout of the device workspace.
// The state of transmitter 0 (E[3], H[3], psiE[6], psiH[6]) is one block
// at E[0]; transmitter k's block starts sstride bytes further per k.
struct Layout {
  size_t status, conv, E[3], H[3], ie[3], psiE[6], psiH[6], sstride, vacc, ring, ring_comp, zero_end;
  int ring_k;
  size_t cm[3], cp[3], pml[3], srcs, jw, amp, rec_start, rec_w, fE, fH, fE32, fH32, norm;
  size_t air_twx, air_twy, air_decE, air_facH, air_work, total;
};

Layout plan(const emm_grid *g, const emm_survey *s, int nsrc = 1);
// Floats of source weights per transmitter (three component boxes, each at
// most the bound of an antenna of survey->src_length on this grid).
size_t source_stride(const emm_grid *g, const emm_survey *s);
int check_survey(const emm_grid *g, const emm_survey *s);

// Derivative axis of CPML array c (0..5): 2*comp + 0 -> (comp+1)%3, 2*comp + 1 -> (comp+2)%3.
inline int psi_axis(int c) { return (c % 2 == 0) ? (c / 2 + 1) % 3 : (c / 2 + 2) % 3; }

// Optional per-launch timing: events before/after the E, volume DTFT and H
// launches of every `every`-th step (4 events per timed step).  With a field
// ring the timed steps are the ends of every (every / ring_k)-th batch, and
// vsteps[q] is the number of steps the volume DTFT launch of sample q
// covered (0: none in it); used counts the samples taken.
struct StepEvents {
  int every = 0;
  int used = 0;
  std::vector<cudaEvent_t> ev;
  std::vector<int> vsteps;
  cudaEvent_t loop[2] = {nullptr, nullptr};  // around the whole time loop
};

// A forward run set up in a workspace: the launch parameters of its steps.
struct Prepared {
  DevParams p;
  Layout L;
  FieldGeom fg;
  dim3 blocks;
  double dt;
  int sms, rd, shape;
};

// Validate, upload the tables, clear the state and compute dt/eps (enqueued
// on cs); fills *out.  Host-detected errors enqueue nothing.
// nsrc transmitters at src_pos ([nsrc][3], host; NULL: the survey's source).
// upload_tables false: the tables are already in the workspace (a repeat of
// an earlier prepare of the same problem); nothing reads host memory after
// the call, so the enqueued work can be captured in a CUDA graph.
// shape: the stencil tile shape of the launches (-1: survey->tile_shape; a
// convergence run takes shape 0).
int prepare_forward(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                    double *rec_out, double *vol_out, cudaStream_t cs, Prepared *out, int nsrc = 1,
                    const double *src_pos = nullptr, bool converge = false, bool upload_tables = true,
                    int shape = -1);
// Enqueue the leapfrog steps n0 .. n1-1 with launch parameters p on grid `blocks`.
cudaError_t run_steps(const Prepared &P, const DevParams &p, dim3 blocks, int n0, int n1, cudaStream_t cs,
                      StepEvents *te);
// Enqueue the Green's-function normalisation of the receivers (and volume).
int finalize_forward(const Prepared &P, const emm_survey *s, double *rec_out, double *vol_out, cudaStream_t cs);

}  // namespace emm
