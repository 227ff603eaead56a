// emm_kernels.cu -- sm_103a kernels of the fictitious-wave FDTD time loop and
// the emm_forward / emm_forward_timed / emm_workspace_size / emm_status
// entry points.
//
// One leapfrog step (Algorithm 1 without the airwave step) is two launches:
//
//   k_update_E<R>  curl H with D- rows and CPML memory (Eq. 14, 22-24), the
//                  electric source at t_{n+1/2}, E += dt/eps (curl H - J)
//                  (Eq. 8); extra CTAs accumulate the receiver DTFT of
//                  H^{n+1/2} (Eq. 25), which this launch only reads.
//   k_update_H<R>  curl E with D+ rows and CPML memory (Eq. 13, 22-24),
//                  H -= dt/mu0 curl E; extra CTAs accumulate the receiver
//                  DTFT of E^{n+1}.
// Runs that need them add dependent launches after the E launch (antenna
// source, air rows above the model, the volume DTFT of E^{n+1} and H^{n+1/2})
// and after the H launch (magnetic source, air rows).
//
// Launch shape: the step is bound by HBM bandwidth, and what the memory
// system needs is many bytes in flight from many CTAs.  A CTA owns a 32 x 8
// column tile over a short run of ZC planes (one thread per column) and the
// grid covers the padded volume thousands of CTAs deep.  On entry one thread
// issues three TMA copies (cp.async.bulk.tensor) that bring the three source
// fields of the tile, with the x, y and z halos their derivatives need, into
// shared memory; meanwhile every thread loads its own samples of the updated
// field and of dt/eps (coalesced 128-byte rows, no reuse) into registers.
// After the copies land, every tap is a shared-memory read at a fixed offset.
// Fields are FP32 in arrays whose rows are padded to 32 samples (rows start on
// 128-byte lines; TMA strides are 16-byte multiples); the receiver DTFT
// accumulates in FP64 and the volume DTFT in compensated FP32 (hi + lo pairs).
// No device transcendentals: every exp/sin/cos comes from FP64 host tables.
//
// The one mbarrier wait of a CTA is bounded (1 s of %globaltimer).  If it
// runs out the status word is set to EMM_ETIMEOUT, the CTA agrees on the
// abort with __syncthreads_or, waits (again bounded) for its copies and
// returns without writing, so no kernel can hang the device.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "emm_internal.h"
#include "emm_tma.cuh"

// Scratch of emm_forward_static: one array per device for the process
// lifetime.  In host code this name only stands for the symbol; its device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char emm_static_scratch[EMM_STATIC_SCRATCH_BYTES];

namespace emm {
namespace {

constexpr int TX = 32;  // tile width (x, one warp)
// Tile shapes, 128 threads each (one per quad of 4 x-adjacent cells):
// shape 0 is 32 (x) by 8 (y) by 2 (z) cells, shape 1 is 32 by 4 by 4.  The
// plain launches use shape 0; the persistent work list takes the shape its
// autotuner picks.
constexpr int kShapes = 2;
__host__ __device__ constexpr int shape_ty(int S) { return S == 1 ? 4 : 8; }  // tile height (y)
__host__ __device__ constexpr int shape_zc(int S) { return S == 1 ? 4 : 2; }  // planes per CTA
constexpr int NT = 128;
static_assert((TX / 4) * shape_ty(0) * shape_zc(0) == NT && (TX / 4) * shape_ty(1) * shape_zc(1) == NT,
              "every tile shape has one thread per quad");
constexpr int XH = 4;   // x halo of the TMA boxes (>= R; keeps box x starts 16-byte aligned)
constexpr int WX = TX + 2 * XH;

// Resident CTAs per SM the register budget is sized for.
__host__ __device__ constexpr int min_ctas(int R) { return R <= 2 ? 5 : 4; }

// Shared-memory tiles of one CTA, for either half-step.  "zf" is the source
// field with z and y halos (Hx / Ex), "xf" the one with z and x halos
// (Hy / Ey), "xy" the one with x and y halos (Hz / Ez).
template <int R, int S = 0>
struct Tiles {
  static constexpr int TY = shape_ty(S), ZC = shape_zc(S);
  static constexpr int ZQ = ZC + 2 * R - 1;  // planes of the z-halo boxes
  static constexpr int YH = TY + 2 * R;      // rows of the y-halo boxes
  static constexpr int ZF = ZQ * YH * TX;
  static constexpr int XF = ZQ * TY * WX;
  static constexpr int XY = ZC * YH * WX;
  static constexpr size_t BYTES = static_cast<size_t>(ZF + XF + XY) * 4;  // the three TMA boxes
  static constexpr int PSI = 6 * NT * 4;  // CPML memory staged per thread: [6 slots][NT] float4
  static constexpr size_t ALL = BYTES + static_cast<size_t>(PSI) * 4;
};
template <int R, int S = 0>
constexpr size_t smem_bytes() { return Tiles<R, S>::ALL + 144; }  // + alignment pad + mbarrier

// Tensor maps of one launch: the three source fields with their boxes.
struct TmaSet {
  CUtensorMap m[3];
};

__device__ __forceinline__ int slab_int(int i, int np, int nb) {
  return i < nb ? i : (i >= np - nb ? nb + np - 1 - i : -1);
}
__device__ __forceinline__ int slab_half(int i, int np, int nb) {
  return i < nb ? i : ((i >= np - 1 - nb && i <= np - 2) ? nb + np - 2 - i : -1);
}

// One warp per (receiver, component): (2R)^3 weighted gather in FP64, warp
// shuffle reduction, then acc += factor * value for every frequency.
// CONV: a convergence run, whose extra warp accumulates the corner DTFT.
template <int R, bool CONV>
__device__ void receiver_dft(const DevParams &p, int comp0, float *const *F, const double *fac, int block,
                             double *rec_acc) {
  constexpr int M = 2 * R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = block * (NT / 32) + warp;
  if (item >= p.nrec * 3) {
    if (CONV && item == p.nrec * 3 && lane < 24) {
      // convergence runs: the corner DTFT, one lane per (corner, component)
      const int q = lane / 3, cc = lane % 3;
      const int i = p.nbe + ((q & 1) ? p.n[0] - 1 : 0), j = p.nbe + ((q & 2) ? p.n[1] - 1 : 0),
                k = p.nbe + ((q & 4) ? p.n[2] - 1 : 0);
      const float *f = cc == 0 ? F[0] : (cc == 1 ? F[1] : F[2]);
      const double v = f[static_cast<size_t>(k) * p.plane + static_cast<size_t>(j) * p.pitch + i];
      double *acc = p.corner + (q * 6 + comp0 + cc) * 2;
      acc[0] += fac[2 * p.conv_f] * v;
      acc[1] += fac[2 * p.conv_f + 1] * v;
    }
    return;
  }
  const int rec = item / 3, c = comp0 + item % 3;
  const int *st = p.rec_start + (rec * 6 + c) * 3;
  const double *w = p.rec_w + static_cast<size_t>(rec * 6 + c) * 3 * M;
  // pick the component without indexing the pointer array (keeps it in registers)
  const int cc = c - comp0;
  const float *f = cc == 0 ? F[0] : (cc == 1 ? F[1] : F[2]);
  double s = 0.0;
  for (int t = lane; t < M * M * M; t += 32) {
    const int q1 = t % M, q2 = (t / M) % M, q3 = t / (M * M);
    const size_t id = (static_cast<size_t>(st[2] + q3) * p.np[1] + (st[1] + q2)) * p.pitch + (st[0] + q1);
    s += w[q1] * w[M + q2] * w[2 * M + q3] * static_cast<double>(f[id]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double *acc = rec_acc + static_cast<size_t>(rec * 6 + c) * p.nf * 2;
    for (int q = 0; q < p.nf; ++q) {
      acc[2 * q] += fac[2 * q] * s;
      acc[2 * q + 1] += fac[2 * q + 1] * s;
    }
  }
}


// ---------------------------------------------------------------------------
// Common CTA prologue: origin of the tile, the TMA copies of the three source
// fields, and the bounded wait for them.  The grid is 3-D: rec_layers z
// layers of receiver CTAs first (so that they run beside the first stencil
// wave instead of trailing the launch), then (tiles_x, tiles_y, tiles_z)
// stencil CTAs.
// ---------------------------------------------------------------------------
// Grid x = transmitter + nsrc * tile: the transmitters of a tile run side by
// side and share its dt/eps reads in L2.
struct Origin {
  int i0, j0, k0, src;
};
// A CTA's place in its problem's launch grid: blockIdx for a launch of one
// problem; for a launch over a work list of problems, the CTA's index
// within its problem's share (see k_update_E_jobs).
struct Blk {
  int x, y, z;
};
__device__ __forceinline__ Blk launch_blk() {
  return Blk{static_cast<int>(blockIdx.x), static_cast<int>(blockIdx.y), static_cast<int>(blockIdx.z)};
}
// MULTI: a batch of transmitters (otherwise transmitter 0 alone, and no
// index arithmetic for it).
template <bool MULTI, int S = 0>
__device__ __forceinline__ Origin origin_of(const DevParams &p, const Blk &b) {
  const int bx = MULTI ? b.x / p.nsrc : b.x;
  return Origin{p.org[0] + bx * TX, p.org[1] + b.y * shape_ty(S), p.org[2] + (b.z - p.rec_layers) * shape_zc(S),
                MULTI ? b.x % p.nsrc : 0};
}
template <bool MULTI>
__device__ __forceinline__ int receiver_block(const DevParams &p, const Blk &b) {
  return (b.z * p.tiles_y + b.y) * p.tiles_x + (MULTI ? b.x / p.nsrc : b.x);
}
template <bool MULTI>
__device__ __forceinline__ int receiver_source(const DevParams &p, const Blk &b) {
  return MULTI ? b.x % p.nsrc : 0;
}

// The state arrays of transmitter src.
struct Fields {
  float *E[3], *H[3], *psiE[6], *psiH[6];
};
template <bool MULTI>
__device__ __forceinline__ Fields fields_of(const DevParams &p, int src) {
  Fields f;
  const size_t o = MULTI ? static_cast<size_t>(src) * p.sstride : 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f.E[a] = p.E[a] + o;
    f.H[a] = p.H[a] + o;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    f.psiE[c] = p.psiE[c] + o;
    f.psiH[c] = p.psiH[c] + o;
  }
  return f;
}

// Thread 0: initialise the CTA's mbarrier (unless a CTA that runs several
// tiles initialised it once already: `phase` > 0 counts the tiles before
// this one) and issue the three copies.  The z-halo boxes start `lead`
// planes from k0 (-R for D-, -R+1 for D+).
template <int R, int S>
__device__ __forceinline__ void issue_tiles(const TmaSet &tm, float *s, uint64_t *bar, const Origin &o, int lead,
                                            unsigned phase) {
  using T = Tiles<R, S>;
  if (phase == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  mbar_expect_tx(bar, static_cast<uint32_t>(T::BYTES));
  tma_load_4d(s, &tm.m[0], bar, o.i0, o.j0 - R, o.k0 + lead, o.src);
  tma_load_4d(s + T::ZF, &tm.m[1], bar, o.i0 - XH, o.j0, o.k0 + lead, o.src);
  tma_load_4d(s + T::ZF + T::XF, &tm.m[2], bar, o.i0 - XH, o.j0 - R, o.k0, o.src);
}

// Wait for the copies: thread 0 (which initialised the barrier and issued
// them) waits on the mbarrier's phase of this tile (parity `phase` & 1),
// bounded; the other threads wait at the CTA barrier that follows, which
// orders the landed tiles before their reads.  False, for the whole CTA, if
// the wait ran out (thread 0 has then set the status word, and the abort
// word of a persistent run, and drained the copies, again bounded).
__device__ __forceinline__ bool tiles_ready(const DevParams &p, uint64_t *bar, unsigned phase) {
  int late = 0;
  if (threadIdx.x == 0 && !mbar_wait_bounded(bar, phase & 1u)) {
    late = 1;
    atomicExch(p.status, EMM_ETIMEOUT);
    if (p.abort) atomicExch(p.abort, 1);
    mbar_wait_bounded(bar, phase & 1u);
  }
  return !__syncthreads_or(late);
}

__device__ __forceinline__ float *smem_tiles(unsigned char *raw) {
  const uint32_t pad = (128u - (smem_u32(raw) & 127u)) & 127u;
  return reinterpret_cast<float *>(raw + pad);
}

// Does the CTA's box meet the bounding box of the source stencils?
template <int S>
__device__ __forceinline__ bool cta_has_source(const SrcDev &sd, const Origin &o) {
  return sd.any && o.i0 + TX > sd.lo[0] && o.i0 <= sd.hi[0] && o.j0 + shape_ty(S) > sd.lo[1] &&
         o.j0 <= sd.hi[1] && o.k0 + shape_zc(S) > sd.lo[2] && o.k0 <= sd.hi[2];
}

// jw: this transmitter's [3][(2R)^3] stencil weights.
template <int R>
__device__ __forceinline__ void source_term(const SrcDev &sd, const float *jw, int c, int i, int j, int k,
                                            float amp, float &curl) {
  constexpr int M = 2 * R;
  if (!sd.on[c]) return;
  const int a = i - sd.start[c][0], bb = j - sd.start[c][1], cc = k - sd.start[c][2];
  if (a >= 0 && a < M && bb >= 0 && bb < M && cc >= 0 && cc < M)
    curl -= amp * jw[(c * M + cc) * M * M + bb * M + a];
}

// ---------------------------------------------------------------------------
// Thread layout of a stencil CTA: the tile is 32 (x) x TY (y) x ZC (z) cells;
// thread t owns the 4 x-adjacent cells ("quad") q = t % 8 of row r = t / 8 % TY
// in plane c = t / (8 TY).  A quad starts on a 16-byte boundary of every field
// row, so its samples move as one float4 and its taps as float4 shared-memory
// reads; derivatives along y and z use paired FP32 FMAs (f32x2).
// ---------------------------------------------------------------------------

struct Quad {
  int q, r, c;   // quad, row, plane inside the tile
  int i, j, k;   // grid coordinates of the first cell
};
template <int S>
__device__ __forceinline__ Quad quad_of(const Origin &o) {
  const int t = threadIdx.x;
  Quad u;
  u.q = t & 7;
  u.r = (t >> 3) % shape_ty(S);
  u.c = t / (8 * shape_ty(S));
  u.i = o.i0 + 4 * u.q;
  u.j = o.j0 + u.r;
  u.k = o.k0 + u.c;
  return u;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// acc[0..3] += coef * v[0..3], two cells per instruction.
struct Acc4 {
  float2 lo, hi;
  __device__ __forceinline__ Acc4() : lo(make_float2(0.f, 0.f)), hi(make_float2(0.f, 0.f)) {}
  __device__ __forceinline__ void fma(float coef, const float4 &v) {
    lo = fma2(make_float2(coef, coef), make_float2(v.x, v.y), lo);
    hi = fma2(make_float2(coef, coef), make_float2(v.z, v.w), hi);
  }
  __device__ __forceinline__ float operator[](int e) const {
    return e == 0 ? lo.x : (e == 1 ? lo.y : (e == 2 ? hi.x : hi.y));
  }
};

__device__ __forceinline__ float get(const float4 &v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ void put(float4 &v, int e, float x) {
  if (e == 0) v.x = x;
  else if (e == 1) v.y = x;
  else if (e == 2) v.z = x;
  else v.w = x;
}

// Shared-memory views of the three tiles (see Tiles), as float4 at quad
// granularity: x is a sample column of the box, a multiple of 4.
template <int R, int S = 0>
struct View {
  using T = Tiles<R, S>;
  const float *s;
  __device__ float4 zf(int pz, int y, int x) const {
    return *reinterpret_cast<const float4 *>(s + (pz * T::YH + y) * TX + x);
  }
  __device__ float4 xf(int pz, int y, int x) const {
    return *reinterpret_cast<const float4 *>(s + T::ZF + (pz * T::TY + y) * WX + x);
  }
  __device__ float4 xy(int pz, int y, int x) const {
    return *reinterpret_cast<const float4 *>(s + T::ZF + T::XF + (pz * T::YH + y) * WX + x);
  }
};

// A row of 12 samples (box columns 4q .. 4q+11) for the x derivatives of a
// quad: cell e of the quad sits at box column 4q + XH + e.
struct Row12 {
  float v[12];
  __device__ __forceinline__ void load(float4 a, float4 b, float4 c) {
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
  }
};

// ---------------------------------------------------------------------------
// CPML memory.  Arrays of derivatives along y and z keep x innermost with the
// field row geometry: y: [np2][2nb][pitch], z: [2nb][np1][pitch] (sample i at
// column i of a row shifted like the fields).  Arrays of derivatives along x
// are [np2][np1][wx] with the near slab at entries 0..nb-1 and the far slab
// at hx + (i - first far sample), hx chosen so that a quad starts on a
// 16-byte boundary there too and no quad of one slab touches the other's
// entries.  The CPML coefficients use the slab entry of Sec. 3.4 (mirrored on
// the far face); only the storage differs.
// ---------------------------------------------------------------------------
struct PsiX {
  int hx, wx, far0;  // storage offset of the far slab, row width, first far sample
};

// Element of the quad's first cell in a y-, z- or x-derivative CPML array.
__device__ __forceinline__ size_t psi_y_at(const DevParams &p, const Quad &u, int sy) {
  return (static_cast<size_t>(u.k) * static_cast<size_t>(2 * p.nb) + static_cast<size_t>(sy)) * p.pitch +
         static_cast<size_t>(u.i);
}
__device__ __forceinline__ size_t psi_z_at(const DevParams &p, const Quad &u, int sz) {
  return (static_cast<size_t>(sz) * p.np[1] + static_cast<size_t>(u.j)) * p.pitch + static_cast<size_t>(u.i);
}
__device__ __forceinline__ size_t psi_x_at(const DevParams &p, const Quad &u, int xs, int wx) {
  return (static_cast<size_t>(u.k) * p.np[1] + static_cast<size_t>(u.j)) * wx + static_cast<size_t>(xs);
}

// Stage this thread's CPML memory (float4 per array) into shared-memory
// slots [slot][thread] with 16-byte asynchronous copies.  Slots: 0 (y) and
// 1 (z) of the first component, 2 (z) and 3 (x) of the second, 4 (x) and
// 5 (y) of the third, matching psi[0..5].  sy, sz: slab entries of the row and
// plane (-1 outside); xs: storage column of the quad's first cell in the
// x-derivative arrays, or -1 if the quad does not touch an x slab.
__device__ __forceinline__ void stage_psi(float4 *ps, float *psi0, float *psi1, float *psi2, float *psi3,
                                          float *psi4, float *psi5, const DevParams &p, const Quad &u, int sy, int sz,
                                          int xs, int wx) {
  float4 *d = ps + threadIdx.x;
  if (sy >= 0) {
    const size_t id = psi_y_at(p, u, sy);
    cp_async16(d, psi0 + id);
    cp_async16(d + 5 * NT, psi5 + id);
  }
  if (sz >= 0) {
    const size_t id = psi_z_at(p, u, sz);
    cp_async16(d + 1 * NT, psi1 + id);
    cp_async16(d + 2 * NT, psi2 + id);
  }
  if (xs >= 0) {
    const size_t id = psi_x_at(p, u, xs, wx);
    cp_async16(d + 3 * NT, psi3 + id);
    cp_async16(d + 4 * NT, psi4 + id);
  }
}

// Storage column of a quad starting at sample i in an x-derivative array, or
// -1 if none of its cells lies in an x slab (slab entries: sample < nb, or
// far0 <= sample <= last).
__device__ __forceinline__ int psi_x_column(int i, int nb, const PsiX &x, int last) {
  if (i < nb) return i;
  if (i + 3 >= x.far0 && i <= last) return x.hx + (i - x.far0);
  return -1;
}

// One CPML update (Eq. 22-23, kappa = 1): psi <- b psi + a d; d + psi.
__device__ __forceinline__ float cpml1(float d, float &psi, float a, float b) {
  psi = fmaf(b, psi, a * d);
  return d + psi;
}

// ---------------------------------------------------------------------------
// E half-step: E^{n+1} = E^n + dt/eps (curl H^{n+1/2} - J^{n+1/2})
// ---------------------------------------------------------------------------
// Is every cell of the CTA inside the CPML-free region where all D- rows
// exist (no slab, no boundary test needed)?
template <int S>
__device__ __forceinline__ bool interior_E(const DevParams &p, const Origin &o, int R) {
  const int m = max(p.nb, R);
  return o.i0 >= m && o.i0 + TX - 1 <= p.np[0] - 1 - m && o.j0 >= m && o.j0 + shape_ty(S) - 1 <= p.np[1] - 1 - m &&
         o.k0 >= m && o.k0 + shape_zc(S) - 1 <= p.np[2] - 1 - m;
}

// One quad of the E update.  FAST: an interior CTA without the source, where
// every validity test is true and every slab test false.
// A quad's FD rows: y and z (one row each) and x (the rows of its 4 cells),
// from the D- (E update) or D+ (H update) tables.  Loaded while the CTA's
// tiles are in flight, so their latency is off the compute phase.
template <int R>
struct Coef {
  float cy[2 * R], cz[2 * R], cx[4][2 * R];
};
template <int R>
__device__ __forceinline__ void load_coef(const float *const *tab, const Quad &u, bool live, Coef<R> &c) {
  constexpr int M = 2 * R;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    c.cy[m] = live ? __ldg(tab[1] + u.j * M + m) : 0.f;
    c.cz[m] = live ? __ldg(tab[2] + u.k * M + m) : 0.f;
  }
  const float4 *c4 = reinterpret_cast<const float4 *>(tab[0] + static_cast<size_t>(live ? u.i : 0) * M);
#pragma unroll
  for (int f = 0; f < M; ++f) {
    const float4 a = live ? __ldg(c4 + f) : float4{};
    c.cx[(4 * f) / M][(4 * f) % M] = a.x;
    c.cx[(4 * f + 1) / M][(4 * f + 1) % M] = a.y;
    c.cx[(4 * f + 2) / M][(4 * f + 2) % M] = a.z;
    c.cx[(4 * f + 3) / M][(4 * f + 3) % M] = a.w;
  }
}

template <int R, bool FAST, int S>
__device__ __forceinline__ void e_quad(const DevParams &p, const Fields &f, const View<R, S> &v, const Quad &u,
                                       const float4 (&e)[3], const float4 (&w)[3], const float4 *ps, int n,
                                       bool src, const SrcDev *sd, const float *jw, const Coef<R> &cf,
                                       float amp) {
  constexpr int M = 2 * R;
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const int q4 = 4 * u.q, t = threadIdx.x;
  const float(&cy)[M] = cf.cy;
  const float(&cz)[M] = cf.cz;
  const float(&cx)[4][M] = cf.cx;
  const bool dm_j = FAST || (u.j >= R && u.j <= np1 - 1 - R);
  const bool dm_k = FAST || (u.k >= R && u.k <= np2 - 1 - R);
  bool dm_i[4];
  int si[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    dm_i[c] = FAST || (u.i + c >= R && u.i + c <= np0 - 1 - R);
    si[c] = FAST ? -1 : slab_int(u.i + c, np0, nb);
  }
  const int sj = FAST ? -1 : slab_int(u.j, np1, nb), sk = FAST ? -1 : slab_int(u.k, np2, nb);
  const int xs = FAST ? -1 : psi_x_column(u.i, nb, PsiX{p.psx_hx[0], p.psx_wx[0], p.psx_far0[0]}, np0 - 1);
  float4 out[3] = {e[0], e[1], e[2]};

  // Ex at (i+1/2, j, k): D-_y Hz - D-_z Hy
  {
    Acc4 dy, dz;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      dy.fma(cy[m], v.xy(u.c, u.r + m, q4 + XH));
      dz.fma(cz[m], v.xf(u.c + m, u.r, q4 + XH));
    }
    float4 py = FAST ? float4{} : ps[0 * NT + t], pz = FAST ? float4{} : ps[1 * NT + t];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(FAST || (u.i + c <= np0 - 2 && dm_j && dm_k))) continue;
      float a = dy[c], b = dz[c];
      if (!FAST) {
        if (sj >= 0) {
          float s = get(py, c);
          a = cpml1(a, s, p.pml[1][sj], p.pml[1][2 * nb + sj]);
          put(py, c, s);
        }
        if (sk >= 0) {
          float s = get(pz, c);
          b = cpml1(b, s, p.pml[2][sk], p.pml[2][2 * nb + sk]);
          put(pz, c, s);
        }
      }
      float curl = a - b;
      if (!FAST && src) source_term<R>(*sd, jw, 0, u.i + c, u.j, u.k, amp, curl);
      put(out[0], c, fmaf(get(w[0], c), curl, get(e[0], c)));
    }
    if (!FAST) {
      if (sj >= 0) *reinterpret_cast<float4 *>(f.psiE[0] + psi_y_at(p, u, sj)) = py;
      if (sk >= 0) *reinterpret_cast<float4 *>(f.psiE[1] + psi_z_at(p, u, sk)) = pz;
    }
  }
  // Ey at (i, j+1/2, k): D-_z Hx - D-_x Hz
  {
    Acc4 dz;
#pragma unroll
    for (int m = 0; m < M; ++m) dz.fma(cz[m], v.zf(u.c + m, u.r + R, q4));
    Row12 hz;
    hz.load(v.xy(u.c, u.r + R, q4), v.xy(u.c, u.r + R, q4 + 4), v.xy(u.c, u.r + R, q4 + 8));
    float4 pz = FAST ? float4{} : ps[2 * NT + t], px = FAST ? float4{} : ps[3 * NT + t];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(FAST || (u.j <= np1 - 2 && dm_i[c] && dm_k))) continue;
      float dx = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) dx = fmaf(cx[c][m], hz.v[XH + c - R + m], dx);
      float b = dz[c];
      if (!FAST) {
        if (sk >= 0) {
          float s = get(pz, c);
          b = cpml1(b, s, p.pml[2][sk], p.pml[2][2 * nb + sk]);
          put(pz, c, s);
        }
        if (si[c] >= 0) {
          float s = get(px, c);
          dx = cpml1(dx, s, p.pml[0][si[c]], p.pml[0][2 * nb + si[c]]);
          put(px, c, s);
        }
      }
      float curl = b - dx;
      if (!FAST && src) source_term<R>(*sd, jw, 1, u.i + c, u.j, u.k, amp, curl);
      put(out[1], c, fmaf(get(w[1], c), curl, get(e[1], c)));
    }
    if (!FAST) {
      if (sk >= 0) *reinterpret_cast<float4 *>(f.psiE[2] + psi_z_at(p, u, sk)) = pz;
      if (xs >= 0)
        *reinterpret_cast<float4 *>(f.psiE[3] + psi_x_at(p, u, xs, p.psx_wx[0])) = px;
    }
  }
  // Ez at (i, j, k+1/2): D-_x Hy - D-_y Hx
  {
    Acc4 dy;
#pragma unroll
    for (int m = 0; m < M; ++m) dy.fma(cy[m], v.zf(u.c + R, u.r + m, q4));
    Row12 hy;
    hy.load(v.xf(u.c + R, u.r, q4), v.xf(u.c + R, u.r, q4 + 4), v.xf(u.c + R, u.r, q4 + 8));
    float4 px = FAST ? float4{} : ps[4 * NT + t], py = FAST ? float4{} : ps[5 * NT + t];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(FAST || (dm_i[c] && dm_j && u.k <= np2 - 2))) continue;
      float dx = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) dx = fmaf(cx[c][m], hy.v[XH + c - R + m], dx);
      float b = dy[c];
      if (!FAST) {
        if (si[c] >= 0) {
          float s = get(px, c);
          dx = cpml1(dx, s, p.pml[0][si[c]], p.pml[0][2 * nb + si[c]]);
          put(px, c, s);
        }
        if (sj >= 0) {
          float s = get(py, c);
          b = cpml1(b, s, p.pml[1][sj], p.pml[1][2 * nb + sj]);
          put(py, c, s);
        }
      }
      float curl = dx - b;
      if (!FAST && src) source_term<R>(*sd, jw, 2, u.i + c, u.j, u.k, amp, curl);
      put(out[2], c, fmaf(get(w[2], c), curl, get(e[2], c)));
    }
    if (!FAST) {
      if (xs >= 0)
        *reinterpret_cast<float4 *>(f.psiE[4] + psi_x_at(p, u, xs, p.psx_wx[0])) = px;
      if (sj >= 0) *reinterpret_cast<float4 *>(f.psiE[5] + psi_y_at(p, u, sj)) = py;
    }
  }
  const size_t id = static_cast<size_t>(u.k) * p.plane + static_cast<size_t>(u.j) * p.pitch + u.i;
#pragma unroll
  for (int a = 0; a < 3; ++a) *reinterpret_cast<float4 *>(f.E[a] + id) = out[a];
}

// One CTA of the E half-step.  CONV: a convergence run (corner DTFT).
// OUT: E^{n+1} goes to p.Eout (E^n stays where it is).
// phase: tiles this CTA ran before this one (0 for a CTA of a launch of its own).
template <int R, bool MULTI, bool CONV, bool OUT, int S = 0>
__device__ __forceinline__ void e_block(const DevParams &p, const TmaSet &tm, const int n, const Blk &b,
                                        unsigned phase = 0) {
  if (b.z < p.rec_layers) {
    const int rs = receiver_source<MULTI>(p, b);
    const Fields f = fields_of<MULTI>(p, rs);
    receiver_dft<R, CONV>(p, 3, f.H, p.fH + static_cast<size_t>(n) * p.nf * 2, receiver_block<MULTI>(p, b),
                    p.rec_acc + static_cast<size_t>(rs) * p.nrec * 6 * p.nf * 2);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  float *s = smem_tiles(smem_raw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(s + Tiles<R, S>::ALL / 4);
  const Origin o = origin_of<MULTI, S>(p, b);
  if (threadIdx.x == 0) issue_tiles<R, S>(tm, s, bar, o, -R, phase);

  const Quad u = quad_of<S>(o);
  Fields f = fields_of<MULTI>(p, o.src);
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const bool live = u.i >= 0 && u.i < np0 && u.j >= 0 && u.j < np1 && u.k >= 0 && u.k < np2;
  // this thread's own samples, loaded while the copies are in flight
  float4 e[3], w[3];
  const size_t id = static_cast<size_t>(u.k) * p.plane + static_cast<size_t>(u.j) * p.pitch + u.i;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    e[a] = live ? *reinterpret_cast<const float4 *>(f.E[a] + id) : float4{};
    w[a] = live ? __ldg(reinterpret_cast<const float4 *>(p.ie[a] + id)) : float4{};
    if (OUT) f.E[a] = p.Eout[a];  // the whole quad is stored, so Eout gets every sample
  }
  const SrcDev *sd = p.srcs + o.src;
  const float *jw = p.jw + static_cast<size_t>(o.src) * 3 * (2 * R) * (2 * R) * (2 * R);
  const bool src = p.src_fused && cta_has_source<S>(*sd, o);
  const bool fast = !src && interior_E<S>(p, o, R);
  float4 *ps = reinterpret_cast<float4 *>(s + Tiles<R, S>::BYTES / 4);
  if (!fast && live)
    stage_psi(ps, f.psiE[0], f.psiE[1], f.psiE[2], f.psiE[3], f.psiE[4], f.psiE[5], p, u, slab_int(u.j, np1, nb),
              slab_int(u.k, np2, nb),
              psi_x_column(u.i, nb, PsiX{p.psx_hx[0], p.psx_wx[0], p.psx_far0[0]}, np0 - 1), p.psx_wx[0]);
  cp_async_commit();
  Coef<R> cf;
  load_coef<R>(p.cm, u, live, cf);
  const float amp = src ? __ldg(p.amp + n) : 0.f;  // the wavelet at t_{n+1/2}, source CTAs only
  cp_async_wait_all();
  if (!tiles_ready(p, bar, phase) || !live) return;
  const View<R, S> v{s};
  if (fast)
    e_quad<R, true, S>(p, f, v, u, e, w, ps, n, false, sd, jw, cf, 0.f);
  else
    e_quad<R, false, S>(p, f, v, u, e, w, ps, n, src, sd, jw, cf, amp);
}

// The E half-step of one problem; every launch of a convergence run returns
// at once after the stop.
template <int R, bool MULTI, bool CONV, bool OUT, int S = 0>
__global__ void __launch_bounds__(NT, min_ctas(R))
    k_update_E(const DevParams p, const __grid_constant__ TmaSet tm, const int n) {
  wait_prior_grid();
  if (CONV && *p.halt) return;  // a convergence run that has stopped
  allow_next_launch();
  e_block<R, MULTI, CONV, OUT, S>(p, tm, n, launch_blk());
}

// ---------------------------------------------------------------------------
// H half-step: H^{n+3/2} = H^{n+1/2} - dt/mu0 curl E^{n+1}
// ---------------------------------------------------------------------------
// Is every cell of the CTA inside the CPML-free region where all D+ rows exist?
template <int S>
__device__ __forceinline__ bool interior_H(const DevParams &p, const Origin &o, int R) {
  const int lo = max(p.nb, R - 1);
  const int hx = min(p.np[0] - 2 - p.nb, p.np[0] - 1 - R), hy = min(p.np[1] - 2 - p.nb, p.np[1] - 1 - R),
            hz = min(p.np[2] - 2 - p.nb, p.np[2] - 1 - R);
  return o.i0 >= lo && o.i0 + TX - 1 <= hx && o.j0 >= lo && o.j0 + shape_ty(S) - 1 <= hy && o.k0 >= lo &&
         o.k0 + shape_zc(S) - 1 <= hz;
}

template <int R, bool FAST, int S>
__device__ __forceinline__ void h_quad(const DevParams &p, const Fields &f, const View<R, S> &v, const Quad &u,
                                       const float4 (&h)[3], const float4 *ps, int n, const Coef<R> &cf) {
  constexpr int M = 2 * R;
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const int q4 = 4 * u.q, t = threadIdx.x;
  const float(&cy)[M] = cf.cy;
  const float(&cz)[M] = cf.cz;
  const float(&cx)[4][M] = cf.cx;
  const bool dp_j = FAST || (u.j >= R - 1 && u.j <= np1 - 1 - R);
  const bool dp_k = FAST || (u.k >= R - 1 && u.k <= np2 - 1 - R);
  bool dp_i[4], in_i[4];
  int si[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    dp_i[c] = FAST || (u.i + c >= R - 1 && u.i + c <= np0 - 1 - R);
    in_i[c] = FAST || (u.i + c < np0);
    si[c] = FAST ? -1 : slab_half(u.i + c, np0, nb);
  }
  const int sj = FAST ? -1 : slab_half(u.j, np1, nb), sk = FAST ? -1 : slab_half(u.k, np2, nb);
  const int xs = FAST ? -1 : psi_x_column(u.i, nb, PsiX{p.psx_hx[1], p.psx_wx[1], p.psx_far0[1]}, np0 - 2);
  const float dt_mu = p.dt_mu;
  float4 out[3] = {h[0], h[1], h[2]};

  // Hx at (i, j+1/2, k+1/2): D+_y Ez - D+_z Ey
  {
    Acc4 dy, dz;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      dy.fma(cy[m], v.xy(u.c, u.r + m + 1, q4 + XH));
      dz.fma(cz[m], v.xf(u.c + m, u.r, q4 + XH));
    }
    float4 py = FAST ? float4{} : ps[0 * NT + t], pz = FAST ? float4{} : ps[1 * NT + t];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(FAST || (in_i[c] && dp_j && dp_k))) continue;
      float a = dy[c], b = dz[c];
      if (!FAST) {
        if (sj >= 0) {
          float s = get(py, c);
          a = cpml1(a, s, p.pml[1][4 * nb + sj], p.pml[1][6 * nb + sj]);
          put(py, c, s);
        }
        if (sk >= 0) {
          float s = get(pz, c);
          b = cpml1(b, s, p.pml[2][4 * nb + sk], p.pml[2][6 * nb + sk]);
          put(pz, c, s);
        }
      }
      put(out[0], c, fmaf(-dt_mu, a - b, get(h[0], c)));
    }
    if (!FAST) {
      if (sj >= 0) *reinterpret_cast<float4 *>(f.psiH[0] + psi_y_at(p, u, sj)) = py;
      if (sk >= 0) *reinterpret_cast<float4 *>(f.psiH[1] + psi_z_at(p, u, sk)) = pz;
    }
  }
  // Hy at (i+1/2, j, k+1/2): D+_z Ex - D+_x Ez
  {
    Acc4 dz;
#pragma unroll
    for (int m = 0; m < M; ++m) dz.fma(cz[m], v.zf(u.c + m, u.r + R, q4));
    Row12 ez;
    ez.load(v.xy(u.c, u.r + R, q4), v.xy(u.c, u.r + R, q4 + 4), v.xy(u.c, u.r + R, q4 + 8));
    float4 pz = FAST ? float4{} : ps[2 * NT + t], px = FAST ? float4{} : ps[3 * NT + t];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(FAST || (dp_i[c] && dp_k))) continue;
      float dx = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) dx = fmaf(cx[c][m], ez.v[XH + c - R + 1 + m], dx);
      float b = dz[c];
      if (!FAST) {
        if (sk >= 0) {
          float s = get(pz, c);
          b = cpml1(b, s, p.pml[2][4 * nb + sk], p.pml[2][6 * nb + sk]);
          put(pz, c, s);
        }
        if (si[c] >= 0) {
          float s = get(px, c);
          dx = cpml1(dx, s, p.pml[0][4 * nb + si[c]], p.pml[0][6 * nb + si[c]]);
          put(px, c, s);
        }
      }
      put(out[1], c, fmaf(-dt_mu, b - dx, get(h[1], c)));
    }
    if (!FAST) {
      if (sk >= 0) *reinterpret_cast<float4 *>(f.psiH[2] + psi_z_at(p, u, sk)) = pz;
      if (xs >= 0)
        *reinterpret_cast<float4 *>(f.psiH[3] + psi_x_at(p, u, xs, p.psx_wx[1])) = px;
    }
  }
  // Hz at (i+1/2, j+1/2, k): D+_x Ey - D+_y Ex
  {
    Acc4 dy;
#pragma unroll
    for (int m = 0; m < M; ++m) dy.fma(cy[m], v.zf(u.c + R - 1, u.r + m + 1, q4));
    Row12 ey;
    ey.load(v.xf(u.c + R - 1, u.r, q4), v.xf(u.c + R - 1, u.r, q4 + 4), v.xf(u.c + R - 1, u.r, q4 + 8));
    float4 px = FAST ? float4{} : ps[4 * NT + t], py = FAST ? float4{} : ps[5 * NT + t];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (!(FAST || (dp_i[c] && dp_j))) continue;
      float dx = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) dx = fmaf(cx[c][m], ey.v[XH + c - R + 1 + m], dx);
      float b = dy[c];
      if (!FAST) {
        if (si[c] >= 0) {
          float s = get(px, c);
          dx = cpml1(dx, s, p.pml[0][4 * nb + si[c]], p.pml[0][6 * nb + si[c]]);
          put(px, c, s);
        }
        if (sj >= 0) {
          float s = get(py, c);
          b = cpml1(b, s, p.pml[1][4 * nb + sj], p.pml[1][6 * nb + sj]);
          put(py, c, s);
        }
      }
      put(out[2], c, fmaf(-dt_mu, dx - b, get(h[2], c)));
    }
    if (!FAST) {
      if (xs >= 0)
        *reinterpret_cast<float4 *>(f.psiH[4] + psi_x_at(p, u, xs, p.psx_wx[1])) = px;
      if (sj >= 0) *reinterpret_cast<float4 *>(f.psiH[5] + psi_y_at(p, u, sj)) = py;
    }
  }
  const size_t id = static_cast<size_t>(u.k) * p.plane + static_cast<size_t>(u.j) * p.pitch + u.i;
#pragma unroll
  for (int a = 0; a < 3; ++a) *reinterpret_cast<float4 *>(f.H[a] + id) = out[a];
}

// The H half-step walks the stencil tiles in the reverse of the E
// half-step's order (CTAs are dispatched in launch-index order): its first
// tiles are those whose E the E launch wrote last and whose H it read last,
// still in L2; and the next E launch starts where this one ends.
template <bool MULTI>
__device__ __forceinline__ Blk reversed_tile(const DevParams &p, const Blk &b) {
  const int bx = p.tiles_x * (MULTI ? p.nsrc : 1);
  return Blk{bx - 1 - b.x, p.tiles_y - 1 - b.y, 2 * p.rec_layers + p.tiles_z - 1 - b.z};
}

// One CTA of the H half-step.
// REV: walk the tiles in reverse launch order (a launch of its own); false
// where a scheduler hands out the tiles itself.
// OUT: H^{n+3/2} goes to p.Hout (H^{n+1/2} stays where it is).
template <int R, bool MULTI, bool CONV, int S = 0, bool REV = true, bool OUT = false>
__device__ __forceinline__ void h_block(const DevParams &p, const TmaSet &tm, const int n, const Blk &blk,
                                        unsigned phase = 0) {
  const Blk b = (!REV || blk.z < p.rec_layers) ? blk : reversed_tile<MULTI>(p, blk);
  if (b.z < p.rec_layers) {
    const int rs = receiver_source<MULTI>(p, b);
    const Fields f = fields_of<MULTI>(p, rs);
    receiver_dft<R, CONV>(p, 0, f.E, p.fE + static_cast<size_t>(n) * p.nf * 2, receiver_block<MULTI>(p, b),
                    p.rec_acc + static_cast<size_t>(rs) * p.nrec * 6 * p.nf * 2);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  float *s = smem_tiles(smem_raw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(s + Tiles<R, S>::ALL / 4);
  const Origin o = origin_of<MULTI, S>(p, b);
  if (threadIdx.x == 0) issue_tiles<R, S>(tm, s, bar, o, 1 - R, phase);

  const Quad u = quad_of<S>(o);
  Fields f = fields_of<MULTI>(p, o.src);
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const bool live = u.i >= 0 && u.i < np0 && u.j >= 0 && u.j < np1 && u.k >= 0 && u.k < np2;
  float4 h[3];
  const size_t id = static_cast<size_t>(u.k) * p.plane + static_cast<size_t>(u.j) * p.pitch + u.i;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h[a] = live ? *reinterpret_cast<const float4 *>(f.H[a] + id) : float4{};
    if (OUT) f.H[a] = p.Hout[a];  // the whole quad is stored, so Hout gets every sample
  }
  const bool fast = interior_H<S>(p, o, R);
  float4 *ps = reinterpret_cast<float4 *>(s + Tiles<R, S>::BYTES / 4);
  if (!fast && live)
    stage_psi(ps, f.psiH[0], f.psiH[1], f.psiH[2], f.psiH[3], f.psiH[4], f.psiH[5], p, u, slab_half(u.j, np1, nb),
              slab_half(u.k, np2, nb),
              psi_x_column(u.i, nb, PsiX{p.psx_hx[1], p.psx_wx[1], p.psx_far0[1]}, np0 - 2), p.psx_wx[1]);
  cp_async_commit();
  Coef<R> cf;
  load_coef<R>(p.cp, u, live, cf);
  cp_async_wait_all();
  if (!tiles_ready(p, bar, phase) || !live) return;
  const View<R, S> v{s};
  if (fast)
    h_quad<R, true, S>(p, f, v, u, h, ps, n, cf);
  else
    h_quad<R, false, S>(p, f, v, u, h, ps, n, cf);
}

template <int R, bool MULTI, bool CONV, int S = 0, bool OUT = false>
__global__ void __launch_bounds__(NT, min_ctas(R))
    k_update_H(const DevParams p, const __grid_constant__ TmaSet tm, const int n) {
  wait_prior_grid();
  if (CONV && *p.halt) return;  // a convergence run that has stopped
  allow_next_launch();
  h_block<R, MULTI, CONV, S, true, OUT>(p, tm, n, launch_blk());
}

// ---------------------------------------------------------------------------
// Work-list launches: the half-steps of several problems (grids of any size,
// one transmitter each, one order R) in one launch.  The launch parameters
// carry every problem's DevParams and its tensor maps for this half-step;
// CTA b of the 1-D grid belongs to the problem j with cta0[j] <= b <
// cta0[j+1] and takes the place of CTA b - cta0[j] of that problem's own
// launch grid (x fastest), so the problems' tails overlap inside one launch
// instead of each draining alone.
// ---------------------------------------------------------------------------
constexpr int kMaxJobs = 16;
struct JobSet {
  TmaSet tm[kMaxJobs];
  DevParams p[kMaxJobs];
  int cta0[kMaxJobs + 1];
  int nt[kMaxJobs];  // a problem whose steps are done returns at once
  int njobs;
};

__device__ __forceinline__ int job_of(const JobSet &J, int b) {
  int j = 0;
  while (j + 1 < J.njobs && b >= J.cta0[j + 1]) ++j;
  return j;
}
__device__ __forceinline__ Blk job_blk(const DevParams &p, int l) {
  const int tx = p.tiles_x, ty = p.tiles_y;
  return Blk{l % tx, (l / tx) % ty, l / (tx * ty)};
}

template <int R>
__global__ void __launch_bounds__(NT, min_ctas(R)) k_update_E_jobs(const __grid_constant__ JobSet J, const int n) {
  wait_prior_grid();
  allow_next_launch();
  const int b = static_cast<int>(blockIdx.x), j = job_of(J, b);
  if (n >= J.nt[j]) return;
  const DevParams &p = J.p[j];
  e_block<R, false, false, false>(p, J.tm[j], n, job_blk(p, b - J.cta0[j]));
}

template <int R>
__global__ void __launch_bounds__(NT, min_ctas(R)) k_update_H_jobs(const __grid_constant__ JobSet J, const int n) {
  wait_prior_grid();
  allow_next_launch();
  const int b = static_cast<int>(blockIdx.x), j = job_of(J, b);
  if (n >= J.nt[j]) return;
  const DevParams &p = J.p[j];
  h_block<R, false, false>(p, J.tm[j], n, job_blk(p, b - J.cta0[j]));
}

// ---------------------------------------------------------------------------
// Persistent work list: every leapfrog step of several problems -- each a
// grid with one transmitter or a batch of them sharing grid and
// conductivity -- in ONE cooperative launch.  The resident CTAs take the E
// half-step's items (every problem's tiles and receiver CTAs) in order from
// a claim counter, meet at a grid barrier, take the H half-step's items,
// meet again, and so on for every step.  An item runs
// the same per-CTA code as the problem's own launch would (e_block /
// h_block), so each problem's results equal its own solve's bit for bit.
// The barrier is an arrival counter in the workspace that only grows: a CTA
// arrives with a release add, then waits with acquire loads for gen * G
// arrivals, at most wait_ns of %globaltimer.  A wait that runs out sets
// EMM_ETIMEOUT and the abort word; every CTA returns at its next barrier.
// Proxy fences on both sides order the generic-proxy field stores of one
// phase before the TMA (async-proxy) reads of the next.
// ---------------------------------------------------------------------------
constexpr int kMaxTasks = 16;
struct PJob {
  TmaSet tmE, tmH;  // source-field maps of the E half-step (H fields) and of the H half-step (E fields)
  DevParams p;
  int bx, by, nt;
};
struct PSet {
  PJob job[kMaxTasks];
  int cta0[kMaxTasks + 1];  // first item of each problem, then the total
  int njobs, nt_max;
  unsigned *bar;            // arrivals so far (zeroed before the launch)
  unsigned long long *claim;  // items claimed so far (zeroed before the launch)
  int *abort;               // nonzero once a wait ran out
  int *status;              // the work list's status word
  unsigned long long wait_ns;
  int skip;                 // testing: the CTA that withholds its first arrival (-1: none)
};
static_assert(sizeof(PSet) <= 32764, "the work list must fit the kernel parameter space");

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned *a, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Barrier number `gen` (1, 2, ...) of the grid; false (for the whole CTA) if
// the CTA is to stop: its wait ran out, another CTA's did, or it is the
// test CTA that withholds its arrival.
__device__ __forceinline__ bool grid_barrier(const PSet &S, unsigned gen) {
  __syncthreads();
  int go = 1;
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (S.skip == static_cast<int>(blockIdx.x) && gen == 1) {
      go = 0;  // leaves without arriving: every other CTA's wait runs out
    } else {
      red_release_add(S.bar, 1u);
      const unsigned target = gen * gridDim.x;
      const unsigned long long t0 = global_ns();
      for (unsigned it = 0;; ++it) {
        if (ld_acquire_u32(S.bar) >= target) break;
        if (*reinterpret_cast<volatile const int *>(S.abort)) {
          go = 0;
          break;
        }
        if ((it & 15u) == 0 && global_ns() - t0 > S.wait_ns) {
          atomicExch(S.status, EMM_ETIMEOUT);
          atomicExch(S.abort, 1);
          go = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  return __syncthreads_and(go) != 0;
}

template <int R, int SH>
__global__ void __launch_bounds__(NT, min_ctas(R)) k_persist(const __grid_constant__ PSet S) {
  __shared__ long long s_b;
  const int total = S.cta0[S.njobs];
  unsigned gen = 0, tiles = 0;  // tiles: stencil tiles this CTA ran (the mbarrier's phase)
  // Items are claimed in order from one counter (the next one while the
  // current one runs), so faster CTAs take more of them.  Every CTA's last
  // claim of a half-step is the one past its end, so half-step k's claims
  // start at k (total + G).
  const long long per_phase = static_cast<long long>(total) + gridDim.x;
  for (int n = 0; n < S.nt_max; ++n) {
    for (int half = 0; half < 2; ++half) {
      const long long base = (2LL * n + half) * per_phase;
      if (threadIdx.x == 0) s_b = static_cast<long long>(atomicAdd(S.claim, 1ull)) - base;
      __syncthreads();
      int j = 0;
      for (;;) {
        const long long bl = s_b;
        if (bl >= total) break;
        const int b = static_cast<int>(bl);
        long long nxt = 0;
        if (threadIdx.x == 0) nxt = static_cast<long long>(atomicAdd(S.claim, 1ull)) - base;
        while (j + 1 < S.njobs && b >= S.cta0[j + 1]) ++j;
        const PJob &J = S.job[j];
        if (n < J.nt) {
          const int l = b - S.cta0[j];
          const Blk blk{l % J.bx, (l / J.bx) % J.by, l / (J.bx * J.by)};
          // the batch form serves single transmitters too (nsrc = 1: the
          // transmitter index is 0 and its state block is the first), so
          // one inlined copy of each half-step is enough
          if (half == 0)
            e_block<R, true, false, false, SH>(J.p, J.tmE, n, blk, tiles);
          else
            h_block<R, true, false, SH>(J.p, J.tmH, n, blk, tiles);
          if (blk.z >= J.p.rec_layers) ++tiles;  // receiver items use no tiles
        }
        __syncthreads();  // the next item reuses the CTA's shared memory
        if (threadIdx.x == 0) s_b = nxt;
        __syncthreads();
      }
      if (!grid_barrier(S, ++gen)) return;
    }
  }
}

// ---------------------------------------------------------------------------
// Wavefront solve: every leapfrog step of one problem in ONE persistent
// launch, with several time steps in flight at once so that a z-layer of
// tiles (all x-y tiles of one run of planes) is brought from DRAM once and
// advanced by `depth` steps while it sits in L2.
//
// Work unit: a layer item (kind, step s, layer l) = the tiles of z-layer l
// for the E half-step (kind 0) or the H half-step (kind 1) of step s, or
// the receiver CTAs of the E half-step (kind 2, H^{s+1/2}) or of the H
// half-step (kind 3, E^{s+1}); each has `T` CTA items.  The host writes the
// layer items in a global order (sweeps of `depth` steps; within a sweep
// the E items of step s0 + d on layer l sit at position l + K d and the H
// items at l + K d + h), and every CTA claims the next CTA item with an
// atomic counter.  A claimed item first waits -- thread 0, acquire loads,
// bounded by wait_ns of %globaltimer -- for the layers it reads to be
// complete, counted by monotone per-layer completion counters:
//   E(s, l) reads H^{s+1/2} of layers l-a .. l+a:  cntH[l'] >= s T
//           (and on receiver layers, R_E(s-1) done:  cntRE >= s RT)
//   H(s, l) reads E^{s+1} of layers l-a .. l+a:    cntE[l'] >= (s+1) T
//           (and on receiver layers, R_H(s) done:  cntRH >= (s+1) RT)
//   R_E(s): cntE[l'] >= (s+1) T on the receiver layers la .. lb
//   R_H(s): cntH[l'] >= s T on the receiver layers
// where a = layers of the z halo and RT the CTA items of one step's
// receivers.  Every dependency lies at an earlier position of the order, so
// the earliest unfinished item can always proceed (all CTAs are resident:
// a cooperative launch).  Completion: proxy fence, release fence, add to
// the item's counter.  Each tile runs e_block / h_block, so the results
// equal emm_forward's bit for bit.
// ---------------------------------------------------------------------------
struct WaveSet {
  TmaSet tmE, tmH;
  DevParams p;
  const unsigned *order;       // layer items: kind | layer << 2 | step << 14
  long long nitems;            // CTA items in all
  int T, RT;                   // CTA items of a layer item; of one step's receivers (rec_layers * T)
  int a, la, lb, L;            // halo layers; receiver layers la .. lb; layers
  unsigned *cntE, *cntH;       // [L] completed tiles per layer (monotone over the steps)
  unsigned *cntR;              // [2]: completed receiver items of the E half-steps (kind 2), of the H half-steps (kind 3)
  unsigned long long *claim;   // next CTA item
  int *abort, *status;
  unsigned long long wait_ns;
};

// Warp 0: wait until every counter a lane names is at least its target
// (lanes 0 .. n-1 each load one, all in flight at once), bounded; false if
// the wait ran out (status and abort set) or another CTA gave up.
__device__ __forceinline__ bool wait_counts(const WaveSet &W, const unsigned *c, unsigned target, int n) {
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    const bool sat = lane >= n || ld_acquire_u32(c) >= target;
    if (__all_sync(0xffffffffu, sat)) return true;
    int stop = 0;
    if (lane == 0) {
      if (*reinterpret_cast<volatile const int *>(W.abort)) {
        stop = 1;
      } else if ((it & 15u) == 0 && global_ns() - t0 > W.wait_ns) {
        atomicExch(W.status, EMM_ETIMEOUT);
        atomicExch(W.abort, 1);
        stop = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    __nanosleep(20);
  }
}

template <int R>
__global__ void __launch_bounds__(NT, min_ctas(R)) k_wave(const __grid_constant__ WaveSet W) {
  __shared__ long long s_idx;
  const DevParams &p = W.p;
  const unsigned T = static_cast<unsigned>(W.T), RT = static_cast<unsigned>(W.RT);
  unsigned tiles = 0;
  if (threadIdx.x == 0) s_idx = static_cast<long long>(atomicAdd(W.claim, 1ull));
  __syncthreads();
  for (;;) {
    const long long idx = s_idx;
    if (idx >= W.nitems) return;
    const unsigned code = W.order[idx / W.T];
    const int t = static_cast<int>(idx % W.T);
    const int kind = static_cast<int>(code & 3u), l = static_cast<int>((code >> 2) & 4095u);
    const int st = static_cast<int>(code >> 14);
    int ok = 1;
    if (threadIdx.x < 32) {
      // the layers this item reads, one counter per lane:
      //   E(s, l): H^{s+1/2} of layers l-a .. l+a (cntH >= s T), and on the
      //            receiver layers the previous step's E receivers (cntR[0] >= s RT)
      //   H(s, l): E^{s+1} of layers l-a .. l+a (cntE >= (s+1) T), and on the
      //            receiver layers this step's H receivers (cntR[1] >= (s+1) RT)
      //   receivers: the receiver layers la .. lb of E^{s+1} (kind 3) or H^{s+1/2} (kind 2)
      const int lane = threadIdx.x;
      const unsigned *c = W.cntE;
      unsigned target = 0;
      int n = 0;
      if (kind < 2) {
        const int lo = max(0, l - W.a), hi = min(W.L - 1, l + W.a);
        const bool rl = l >= W.la && l <= W.lb;
        n = hi - lo + 1 + (rl ? 1 : 0);
        if (lane <= hi - lo) {
          c = (kind == 0 ? W.cntH : W.cntE) + lo + lane;
          target = static_cast<unsigned>(kind == 0 ? st : st + 1) * T;
        } else {
          c = W.cntR + (kind == 0 ? 0 : 1);
          target = static_cast<unsigned>(kind == 0 ? st : st + 1) * RT;
        }
      } else {
        n = W.lb - W.la + 1;
        c = (kind == 3 ? W.cntE : W.cntH) + W.la + min(lane, n - 1);
        target = static_cast<unsigned>(kind == 3 ? st + 1 : st) * T;
      }
      ok = wait_counts(W, c, target, n) ? 1 : 0;
      if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    if (!__syncthreads_and(ok)) return;
    // the next item is claimed now; its index is needed only after this one
    unsigned long long nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(W.claim, 1ull);
    const Blk b{t % p.tiles_x, t / p.tiles_x, kind >= 2 ? l : p.rec_layers + l};
    if (kind == 0 || kind == 2)
      e_block<R, false, false, false, 0>(p, W.tmE, st, b, tiles);
    else
      h_block<R, false, false, 0, false>(p, W.tmH, st, b, tiles);
    if (kind < 2) ++tiles;
    __syncthreads();
    if (threadIdx.x == 0) {
      // receivers count in cntR[0] (kind 3, E^{s+1}) and cntR[1] (kind 2, H^{s+1/2})
      unsigned *c = kind == 0 ? W.cntE + l : kind == 1 ? W.cntH + l : W.cntR + (kind == 3 ? 0 : 1);
      red_release_add(c, 1u);
      s_idx = static_cast<long long>(nxt);
    }
    __syncthreads();
  }
}

// Sources the stencil kernels do not inject themselves, one thread per
// (transmitter, component, box sample):
//   FIELD 0, after the E launch of step n: an electric antenna,
//     E -= dt/eps J with J = amp(t_{n+1/2}) dir_c w / V;
//   FIELD 1, after the H launch: a magnetic dipole or antenna,
//     mu dH/dt = -(curl E + M) (Eq. 1 in the time domain), so
//     H -= dt/mu0 M with M = amp(t_{n+1}) dir_c w / V.
template <bool MULTI, int FIELD>
__global__ void k_inject(const DevParams p, const int n) {
  wait_prior_grid();
  if (p.halt && *p.halt) return;  // a convergence run that has stopped
  allow_next_launch();
  const size_t per = p.jstride, cv = per / 3;
  const size_t t = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= static_cast<size_t>(p.nsrc) * per) return;
  const int src = static_cast<int>(t / per), c = static_cast<int>((t % per) / cv);
  const int node = static_cast<int>(t % cv);
  const SrcDev &sd = p.srcs[src];
  const int bx = sd.box[c][0], by = sd.box[c][1], bz = sd.box[c][2];
  if (!sd.on[c] || node >= bx * by * bz) return;
  const int q1 = node % bx, q2 = (node / bx) % by, q3 = node / (bx * by);
  const Fields f = fields_of<MULTI>(p, src);
  const size_t id = static_cast<size_t>(sd.start[c][2] + q3) * p.plane +
                    static_cast<size_t>(sd.start[c][1] + q2) * p.pitch + (sd.start[c][0] + q1);
  const float a = __ldg(p.amp + n) * p.jw[static_cast<size_t>(src) * per + sd.woff[c] + node];
  if (FIELD == 0) {
    float *E = c == 0 ? f.E[0] : (c == 1 ? f.E[1] : f.E[2]);
    E[id] = fmaf(-p.ie[c][id], a, E[id]);
  } else {
    float *H = c == 0 ? f.H[0] : (c == 1 ? f.H[1] : f.H[2]);
    H[id] = fmaf(-p.dt_mu, a, H[id]);
  }
}

// ---- Air above the model (Sec. 3.3) ---------------------------------------
// KIND 0, after the E launch: the E_x, E_y interface rows continued to the
// rd - 1 integer rows above; KIND 1, after the H launch: the H_z interface
// row to H_x, H_y on the rd half rows above.  The 2-D DFT of the padded x-y
// plane and its inverse are four passes of 1-D transforms:
//   MODE 0 (rows):     T[c][j][q] = sum_i f_c(i, j) w0^{q i}
//   MODE 1 (columns):  F[c][k][q] = sum_j w1^{k j} T[c][j][q]
//   MODE 2 (inverse columns, times the continuation factor of output o):
//                      U[o][j][q] = sum_k conj(w1^{j k}) F[c(o)][k][q] fac_o[k][q]
//   MODE 3 (inverse rows, real part, into the field row of output o):
//                      out_o(i, j) = Re sum_q U[o][j][q] conj(w0^{q i}) / (N0 N1)
// with w0 = e^{-2 pi i / N0}, w1 = e^{-2 pi i / N1}.  One CTA per line
// (grid x = line, z = transmitter): the line is gathered into shared memory
// and transformed by a mixed-radix Stockham FFT (radix 4 while 4 divides
// the rest of N, then its smallest prime factors; any N), one thread per
// output sample of each stage, with the roots of unity (tabulated in FP64
// on the host) in shared memory.
constexpr int AFT = 256;  // threads of an air transform CTA

// One Stockham stage of a length-N transform: radix r after sub-transforms
// of length Ns.  Output o = (t / Ns) Ns r + p Ns + k (k < Ns, p < r) is
//   sum_q in[t + q N / r] W^{q (k + p Ns) N / (Ns r)},  t = (o / (Ns r)) Ns + k,
// W = e^{-2 pi i / N} (conjugated for the inverse).
template <bool INV>
__device__ __forceinline__ void fft_stage(const float2 *in, float2 *out, const float2 *W, int N, int Ns, int r) {
  const int span = Ns * r, step = N / span, m = N / r;
  for (int o = threadIdx.x; o < N; o += AFT) {
    const int blk = o / span, w = o % span, pp = w / Ns, k = w % Ns, t = blk * Ns + k;
    const int e = (k + pp * Ns) * step;  // W exponent of q = 1
    float2 acc = in[t];
    int x = 0;
    for (int q = 1; q < r; ++q) {
      x += e;
      if (x >= N) x -= N;
      const float2 a = in[t + q * m], wq = W[x];
      const float wy = INV ? -wq.y : wq.y;
      acc.x = fmaf(a.x, wq.x, fmaf(-a.y, wy, acc.x));
      acc.y = fmaf(a.x, wy, fmaf(a.y, wq.x, acc.y));
    }
    out[o] = acc;
  }
  __syncthreads();
}

// Transforms the line in b0 over the buffers b0, b1; returns the buffer
// that holds the result.
template <bool INV>
__device__ __forceinline__ float2 *fft_line(float2 *b0, float2 *b1, const float2 *W, int N) {
  int rest = N, Ns = 1;
  while (rest > 1) {
    int r = rest % 4 == 0 ? 4 : 0;
    if (!r) {
      r = 2;
      while (rest % r) r = r == 2 ? 3 : r + 2;
    }
    fft_stage<INV>(b0, b1, W, N, Ns, r);
    float2 *t = b0;
    b0 = b1;
    b1 = t;
    Ns *= r;
    rest /= r;
  }
  return b0;
}

// Shared memory: the N roots of unity and two line buffers.
// The roots of unity and the continuation factors are set-up tables, so a
// CTA stages them before griddepcontrol.wait (overlapping the previous
// launch's drain); the lines themselves, written by the launch before, are
// gathered after it.
template <int MODE, bool MULTI, int KIND>
__global__ void __launch_bounds__(AFT) k_air_fft(const DevParams p) {
  extern __shared__ float2 air_sm[];
  const int N0 = p.np[0], N1 = p.np[1], rd = p.air_rd, src = static_cast<int>(blockIdx.z);
  const int N = (MODE == 0 || MODE == 3) ? N0 : N1;
  const int ln = static_cast<int>(blockIdx.x);  // line: MODE 0 c N1 + j; 1 c N0 + q; 2 o N0 + q; 3 o N1 + j
  const size_t plane = static_cast<size_t>(N0) * N1;
  float2 *Ws = air_sm, *b0 = air_sm + N, *b1 = b0 + N;
  const float2 *W = (MODE == 0 || MODE == 3) ? p.air_twx : p.air_twy;
  for (int i = threadIdx.x; i < N; i += AFT) {
    Ws[i] = W[i];
    if (MODE == 2) {  // the continuation factor of this line's output, sample k = i
      const int o = ln / N0, q = ln % N0, r2 = o / 2;
      const size_t fi = static_cast<size_t>(i) * N0 + q;
      b1[i] = KIND == 0 ? make_float2(p.air_decE[r2 * plane + fi], 0.f)
                        : p.air_facH[(static_cast<size_t>(o % 2) * rd + r2) * plane + fi];
    }
  }
  wait_prior_grid();
  if (p.halt && *p.halt) return;
  allow_next_launch();
  const Fields f = fields_of<MULTI>(p, src);
  float2 *T = p.air_T + static_cast<size_t>(src) * 3 * plane;
  float2 *F = p.air_F + static_cast<size_t>(src) * 3 * plane;
  float2 *U = p.air_U + static_cast<size_t>(src) * 2 * rd * plane;
  for (int i = threadIdx.x; i < N; i += AFT) {
    float2 v;
    if (MODE == 0) {
      const int c = ln / N1, j = ln % N1;
      const float *fc = KIND == 0 ? (c == 0 ? f.E[0] : f.E[1]) : f.H[2];
      v = make_float2(fc[static_cast<size_t>(p.air_ks) * p.plane + static_cast<size_t>(j) * p.pitch + i], 0.f);
    } else if (MODE == 1) {
      const int c = ln / N0, q = ln % N0;
      v = T[(static_cast<size_t>(c) * N1 + i) * N0 + q];
    } else if (MODE == 2) {
      const int o = ln / N0, q = ln % N0, comp = KIND == 0 ? o % 2 : 0;
      const float2 x = F[(static_cast<size_t>(comp) * N1 + i) * N0 + q], g = b1[i];  // b1: this thread's own factor
      v = KIND == 0 ? make_float2(x.x * g.x, x.y * g.x) : make_float2(x.x * g.x - x.y * g.y, x.x * g.y + x.y * g.x);
    } else {
      v = U[static_cast<size_t>(ln) * N0 + i];  // ln = o N1 + j
    }
    b0[i] = v;
  }
  __syncthreads();
  const float2 *res = fft_line<(MODE >= 2)>(b0, b1, Ws, N);
  const float scale = 1.f / (static_cast<float>(N0) * static_cast<float>(N1));
  for (int i = threadIdx.x; i < N; i += AFT) {
    const float2 v = res[i];
    if (MODE == 0) {
      T[static_cast<size_t>(ln) * N0 + i] = v;  // ln = c N1 + j
    } else if (MODE == 1) {
      const int c = ln / N0, q = ln % N0;
      F[(static_cast<size_t>(c) * N1 + i) * N0 + q] = v;
    } else if (MODE == 2) {
      const int o = ln / N0, q = ln % N0;
      U[(static_cast<size_t>(o) * N1 + i) * N0 + q] = v;
    } else {
      const int o = ln / N1, j = ln % N1, r2 = o / 2, d = o % 2;
      float *out = KIND == 0 ? (d == 0 ? f.E[0] : f.E[1]) : (d == 0 ? f.H[0] : f.H[1]);
      out[static_cast<size_t>(p.air_ks - 1 - r2) * p.plane + static_cast<size_t>(j) * p.pitch + i] = v.x * scale;
    }
  }
}

// Steps of fields a solve keeps for its volume DTFT (see ring_depth).
constexpr int kRing = EMM_VOLUME_RING;

// Slot s of the field ring, component c (0..2 E, 3..5 H); see DevParams.
inline const float *ring_field(const DevParams &p, int s, int c) {
  if (s == 0) return c < 3 ? p.E[c] : p.H[c - 3];
  return p.ring + (static_cast<size_t>(s - 1) * 6 + c) * p.ring_comp;
}

// The fields one volume-DTFT launch reads: for its step b0 + s, component c,
// E^{b0+s+1} (c < 3) or H^{b0+s+1/2} (c >= 3).
struct VolFields {
  const float *f[kRing][6];
};

// Pairs of FP32 values (the real and imaginary parts) held in one 64-bit
// register, for the packed FP32x2 instructions.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(r));
  return d;
}

// (hi, lo) += w * (v, v) for two independent sums at once: per lane the
// product x = w v rounded on its own, then the error-free sum of Knuth's
// TwoSum: t = hi + x, b = t - hi, e = (hi - (t - b)) + (x - b); hi = t,
// lo += e.
__device__ __forceinline__ void two_sum_mul_add2(unsigned long long &hi, unsigned long long &lo,
                                                 unsigned long long w, unsigned long long vv) {
  asm("{\n .reg .b64 x, t, b, u, e;\n"
      " mul.rn.f32x2 x, %2, %3;\n"
      " add.rn.f32x2 t, %0, x;\n sub.rn.f32x2 b, t, %0;\n sub.rn.f32x2 u, t, b;\n sub.rn.f32x2 u, %0, u;\n"
      " sub.rn.f32x2 e, x, b;\n add.rn.f32x2 e, u, e;\n add.rn.f32x2 %1, %1, e;\n mov.b64 %0, t;\n}\n"
      : "+l"(hi), "+l"(lo)
      : "l"(w), "l"(vv));
}

// Volume DTFT (Eq. 25 on every interior sample) of the cnt <= kRing steps
// b0 .. b0+cnt-1, launched after the E launch of the last of them (and the
// source and air launches that follow it): for each step n the terms of
// E^{n+1} and H^{n+1/2}, six components and every frequency, acc += factor *
// value in compensated FP32 (hi + lo pairs of the real and imaginary parts),
// added to each accumulator step after step.  Each accumulator is read and
// written once per launch.  One thread per interior sample (i fastest) and
// component: grid x covers a z plane of samples, y the planes, z the six
// components.
__global__ void __launch_bounds__(256) k_volume_dft(const DevParams p, const __grid_constant__ VolFields vf,
                                                    const int b0, const int cnt) {
  wait_prior_grid();
  if (p.halt && *p.halt) return;  // a convergence run that has stopped
  allow_next_launch();
  const unsigned n0 = static_cast<unsigned>(p.n[0]), nplane = n0 * static_cast<unsigned>(p.n[1]);
  const unsigned l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nplane) return;
  const int c = blockIdx.z, kk = blockIdx.y;
  const int ii = static_cast<int>(l % n0), jj = static_cast<int>(l / n0);
  const size_t nint = static_cast<size_t>(nplane) * p.n[2];
  const size_t lin = static_cast<size_t>(kk) * nplane + l;
  const size_t id = static_cast<size_t>(kk + p.nbe) * p.plane + static_cast<size_t>(jj + p.nbe) * p.pitch + (ii + p.nbe);
  unsigned long long vv[kRing];  // (value, value) of each step
#pragma unroll
  for (int s = 0; s < kRing; ++s)
    if (s < cnt) {
      const float x = __ldg(vf.f[s][c] + id);
      vv[s] = pack2(x, x);
    }
  // factors (re, im) of step b0 + s, frequency f at fac[s * nf + f]
  const unsigned long long *fac =
      reinterpret_cast<const unsigned long long *>(c < 3 ? p.fE32 : p.fH32) + static_cast<size_t>(b0) * p.nf;
  constexpr int FG = 4;  // frequencies per round of accumulator loads
  for (int f0 = 0; f0 < p.nf; f0 += FG) {
    float4 *a = p.vacc + (static_cast<size_t>(c) * p.nf + f0) * nint + lin;
    unsigned long long hi[FG], lo[FG];  // (re, im) pairs
#pragma unroll
    for (int g = 0; g < FG; ++g)
      if (f0 + g < p.nf) {
        const float4 t = __ldcs(a + g * nint);  // streamed: touched once per launch
        hi[g] = pack2(t.x, t.z);
        lo[g] = pack2(t.y, t.w);
      }
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
      if (s < cnt) {
#pragma unroll
        for (int g = 0; g < FG; ++g)
          if (f0 + g < p.nf) two_sum_mul_add2(hi[g], lo[g], __ldg(fac + s * p.nf + f0 + g), vv[s]);
      }
    }
#pragma unroll
    for (int g = 0; g < FG; ++g)
      if (f0 + g < p.nf) {
        const float2 h = unpack2(hi[g]), l = unpack2(lo[g]);
        __stcs(a + g * nint, make_float4(h.x, l.x, h.y, l.y));
      }
  }
}

// The launch of k_volume_dft for steps b0 .. b0+cnt-1, slot(step, c) giving
// the field of each.
template <typename Slot>
cudaError_t launch_volume(const DevParams &p, int b0, int cnt, Slot slot, cudaStream_t st) {
  VolFields vf{};
  for (int s = 0; s < cnt; ++s)
    for (int c = 0; c < 6; ++c) vf.f[s][c] = slot(b0 + s, c);
  const unsigned nplane = static_cast<unsigned>(p.n[0]) * static_cast<unsigned>(p.n[1]);
  if (p.n[2] > 65535 || static_cast<size_t>(p.n[0]) * p.n[1] > (1u << 31)) return cudaErrorInvalidValue;
  const dim3 grid((nplane + 255) / 256, static_cast<unsigned>(p.n[2]), 6);
  return launch_dependent(k_volume_dft, grid, dim3(256), 0, st, p, vf, b0, cnt);
}

// dt/eps on the padded grid from the interior staggered conductivity, with
// the pads replicating the edge (model extension, Sec. 3.8), and the input
// check (finite, positive, >= sigma_min).
__global__ void k_prepare(const float *__restrict__ sigma, float *ie0, float *ie1, float *ie2, int n0,
                          int n1, int n2, int np0, int np1, int np2, int pitch, int xshift, int nbe,
                          double two_w0_dt, double sigma_min, int *status) {
  const size_t cells = static_cast<size_t>(pitch) * np1 * np2;  // including the row padding
  const size_t nint = static_cast<size_t>(n0) * n1 * n2;
  float *ie[3] = {ie0, ie1, ie2};
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < 3 * cells;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(t / cells);
    const size_t r = t % cells;
    const int i = static_cast<int>(r % pitch) - xshift, j = static_cast<int>((r / pitch) % np1),
              k = static_cast<int>(r / (static_cast<size_t>(pitch) * np1));
    if (i < 0 || i >= np0) {  // row padding: defined zeros, never used
      ie[c][r] = 0.f;
      continue;
    }
    const int a = min(max(i - nbe, 0), n0 - 1), b = min(max(j - nbe, 0), n1 - 1),
              cc = min(max(k - nbe, 0), n2 - 1);
    const float s = sigma[c * nint + (static_cast<size_t>(cc) * n1 + b) * n0 + a];
    const size_t o = r;
    if (!(s > 0.f) || !isfinite(s) || static_cast<double>(s) < sigma_min) {
      atomicExch(status, EMM_EDEVICE);
      ie[c][o] = 0.f;
    } else {
      ie[c][o] = static_cast<float>(two_w0_dt / static_cast<double>(s));
    }
  }
}

// Green's functions at receivers, in place: G = norm[c][f] * acc  (Eq. 7)
__global__ void k_finalize_rec(double *acc, const double *norm, int nrec, int nf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrec * 6 * nf) return;
  const int f = t % nf, c = (t / nf) % 6;
  const double nr = norm[(c < 3 ? 0 : 1) * nf * 2 + 2 * f], ni = norm[(c < 3 ? 0 : 1) * nf * 2 + 2 * f + 1];
  const double ar = acc[2 * t], ai = acc[2 * t + 1];
  acc[2 * t] = nr * ar - ni * ai;
  acc[2 * t + 1] = nr * ai + ni * ar;
}

// Volume Green's functions: vol[c][f][..] = norm[c][f] * (hi + lo)
__global__ void k_finalize_vol(const float4 *vacc, double *vol, const double *norm, size_t nint, int nf) {
  const size_t total = 6 * static_cast<size_t>(nf) * nint;
  for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < total;
       t += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int cf = static_cast<int>(t / nint);
    const int f = cf % nf, c = cf / nf;
    const double nr = norm[(c < 3 ? 0 : 1) * nf * 2 + 2 * f], ni = norm[(c < 3 ? 0 : 1) * nf * 2 + 2 * f + 1];
    const float4 a = vacc[t];
    const double ar = static_cast<double>(a.x) + a.y, ai = static_cast<double>(a.z) + a.w;
    vol[2 * t] = nr * ar - ni * ai;
    vol[2 * t + 1] = nr * ai + ni * ar;
  }
}

// Corner test of a convergence run (Sec. 4.1), after step `it`: with
// init, remember the corner DTFT; otherwise the run has converged when, at
// each of the 8 corners, the change of the corner DTFT (six components,
// lowest frequency) since the last check is at most 1e-5 of its current
// value and that value is nonzero.  Then *halt = it + 1, the steps to keep.
// host (mapped host memory): [0] the last step checked, [1] *halt.
__global__ void k_corner_check(double *corner, int *halt, volatile int *host, int it, int init) {
  if (*halt) return;  // stopped at an earlier check: the look-ahead chunk changed nothing
  const int lane = threadIdx.x;
  double *prev = corner + 8 * 6 * 2;
  bool ok = true;
  if (!init && lane < 8) {
    double dn = 0.0, un = 0.0;
    for (int c = 0; c < 6; ++c) {
      const double *a = corner + (lane * 6 + c) * 2, *b = prev + (lane * 6 + c) * 2;
      const double dr = a[0] - b[0], di = a[1] - b[1];
      dn += dr * dr + di * di;
      un += a[0] * a[0] + a[1] * a[1];
    }
    ok = un > 0.0 && !(sqrt(dn) > 1e-5 * sqrt(un));
  }
  const bool all = __all_sync(0xffffffffu, ok);
  for (int t = lane; t < 8 * 6 * 2; t += 32) prev[t] = corner[t];
  if (lane == 0) {
    if (!init && all) {
      *halt = it + 1;
      host[1] = it + 1;
    }
    host[0] = it;
    __threadfence_system();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side of emm_forward
// ---------------------------------------------------------------------------
FieldGeom field_geom(const emm_grid *g, int shape) {
  FieldGeom f{};
  const int lo = std::max(g->nb, g->rd);
  const int lo4 = lo & ~3;
  const int step[3] = {TX, shape_ty(shape), shape_zc(shape)};
  const int first[3] = {lo4, lo, lo};
  for (int a = 0; a < 3; ++a) {
    f.org[a] = first[a] - step[a] * ((first[a] + step[a] - 1) / step[a]);
    f.tiles[a] = (g->ax[a].npad - f.org[a] + step[a] - 1) / step[a];
  }
  f.xshift = -f.org[0];
  f.pitch = (g->ax[0].npad + f.xshift + 31) / 32 * 32;
  // Far slab of the x-derivative CPML arrays: stored from hx = (first far
  // sample) mod 4 above the near slab's last quad, so quads stay 16-byte
  // aligned and never overlap the near slab's entries.
  const int np0 = g->ax[0].npad, nb = g->nb, nb4 = (nb + 3) / 4 * 4;
  const int far0[2] = {np0 - nb, np0 - 1 - nb};
  for (int h = 0; h < 2; ++h) {
    f.psx_far0[h] = far0[h];
    f.psx_hx[h] = nb4 + 4 + (far0[h] & 3);
    f.psx_wx[h] = (f.psx_hx[h] + nb + 3 + 3) / 4 * 4;
  }
  return f;
}

// Elements of one CPML memory array (layouts in the kernels' comment).
size_t psi_elems(const emm_grid *g, int axis, int half) {
  const FieldGeom f = field_geom(g);
  const size_t nb2 = 2 * static_cast<size_t>(g->nb);
  const size_t p1 = g->ax[1].npad, p2 = g->ax[2].npad;
  if (axis == 0) return p2 * p1 * static_cast<size_t>(f.psx_wx[half]);
  if (axis == 1) return p2 * nb2 * static_cast<size_t>(f.pitch);
  return nb2 * p1 * static_cast<size_t>(f.pitch);
}


// Per axis, an antenna of length L along dir spans at most
// ceil(L |dir_a| / h_min) + 1 sample intervals between its sub-dipoles'
// stencil starts, h_min the smallest spacing of the axis (nodes or half
// nodes); each stencil adds 2rd samples.
static void source_box_bound(const emm_grid *g, const emm_survey *s, int ext[3]) {
  const double dir[3] = {std::cos(s->src_dip) * std::cos(s->src_az), std::cos(s->src_dip) * std::sin(s->src_az),
                         std::sin(s->src_dip)};
  const int m = 2 * g->rd;
  for (int a = 0; a < 3; ++a) {
    ext[a] = m;
    if (!(s->src_length > 0)) continue;
    const Axis &ax = g->ax[a];
    double h = 1e300;
    for (size_t i = 0; i + 1 < ax.X.size(); ++i) h = std::min(h, ax.X[i + 1] - ax.X[i]);
    for (size_t i = 0; i + 1 < ax.Xh.size(); ++i) h = std::min(h, ax.Xh[i + 1] - ax.Xh[i]);
    ext[a] = m + static_cast<int>(std::ceil(s->src_length * std::fabs(dir[a]) / h)) + 2;
  }
}

size_t source_stride(const emm_grid *g, const emm_survey *s) {
  int ext[3];
  source_box_bound(g, s, ext);
  return 3 * static_cast<size_t>(ext[0]) * ext[1] * ext[2];
}

// Steps of fields a solve keeps for its volume DTFT: a one-transmitter solve
// with the volume DTFT keeps kRing (its half-steps write into a ring of field
// slots and one DTFT launch adds kRing steps' terms to each accumulator, which
// is then read and written once per kRing steps instead of every step); any
// other solve keeps its fields in place.
int ring_depth(const emm_survey *s, int nsrc) { return (s->volume && nsrc == 1) ? kRing : 1; }

Layout plan(const emm_grid *g, const emm_survey *s, int nsrc) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t cells = static_cast<size_t>(field_geom(g).pitch) * g->ax[1].npad * g->ax[2].npad;
  const size_t nint = static_cast<size_t>(g->ax[0].n) * g->ax[1].n * g->ax[2].n;
  const size_t m = 2 * static_cast<size_t>(g->rd), nf = s->nfreq;
  const size_t nt = s->nt > 0 ? s->nt : 1, nrec = s->nrec > 0 ? s->nrec : 1;
  L.status = take(sizeof(int));
  L.conv = take((2 * 8 * 6 * 2) * sizeof(double) + 2 * sizeof(int));  // corners, last check, stop word
  // transmitter 0's state block; transmitters 1 .. nsrc-1 follow it
  const size_t b0 = off;
  for (int c = 0; c < 3; ++c) L.E[c] = take(cells * 4);
  for (int c = 0; c < 3; ++c) L.H[c] = take(cells * 4);
  for (int c = 0; c < 6; ++c) L.psiE[c] = take(psi_elems(g, psi_axis(c), 0) * 4);
  for (int c = 0; c < 6; ++c) L.psiH[c] = take(psi_elems(g, psi_axis(c), 1) * 4);
  L.sstride = off - b0;
  off += static_cast<size_t>(nsrc > 1 ? nsrc - 1 : 0) * L.sstride;
  L.vacc = take(s->volume ? 6 * nf * nint * sizeof(float4) : 0);
  // field ring of a one-transmitter solve with the volume DTFT: slots 1 ..
  // ring_k-1 of E and H (slot 0 is the state's), zeroed like the state
  L.ring_k = ring_depth(s, nsrc);
  L.ring_comp = align_up(cells * 4);
  L.ring = take(static_cast<size_t>(L.ring_k - 1) * 6 * L.ring_comp);
  L.zero_end = off;
  for (int c = 0; c < 3; ++c) L.ie[c] = take(cells * 4);
  // air: work planes T, F (3 components) and U (2 rd outputs) per transmitter
  const size_t plane2 = static_cast<size_t>(g->ax[0].npad) * g->ax[1].npad;
  L.air_work = take(s->airwave ? static_cast<size_t>(nsrc) * (6 + 2 * g->rd) * plane2 * 8 : 0);
  // FD rows; the x tables run on to a whole field row (zero rows past npad),
  // because the kernels read the rows of all four cells of a quad at once
  const size_t xrows = std::max<size_t>(g->ax[0].npad, field_geom(g).pitch);
  for (int a = 0; a < 3; ++a) L.cm[a] = take((a == 0 ? xrows : g->ax[a].npad) * m * 4);
  for (int a = 0; a < 3; ++a) L.cp[a] = take((a == 0 ? xrows : g->ax[a].npad) * m * 4);
  for (int a = 0; a < 3; ++a) L.pml[a] = take(8 * static_cast<size_t>(g->nb) * 4);
  L.srcs = take(static_cast<size_t>(nsrc) * sizeof(SrcDev));
  L.jw = take(static_cast<size_t>(nsrc) * source_stride(g, s) * 4);
  L.amp = take(nt * 4);
  L.rec_start = take(nrec * 18 * sizeof(int));
  L.rec_w = take(nrec * 18 * m * sizeof(double));
  L.fE = take(nt * nf * 2 * sizeof(double));
  L.fH = take(nt * nf * 2 * sizeof(double));
  L.fE32 = take(nt * nf * 2 * sizeof(float));
  L.fH32 = take(nt * nf * 2 * sizeof(float));
  L.norm = take(2 * nf * 2 * sizeof(double));
  // air: twiddles and continuation factors
  L.air_twx = take(s->airwave ? static_cast<size_t>(g->ax[0].npad) * 8 : 0);
  L.air_twy = take(s->airwave ? static_cast<size_t>(g->ax[1].npad) * 8 : 0);
  L.air_decE = take(s->airwave ? static_cast<size_t>(g->rd - 1) * plane2 * 4 : 0);
  L.air_facH = take(s->airwave ? 2 * static_cast<size_t>(g->rd) * plane2 * 8 : 0);
  L.total = off;
  return L;
}

int check_survey(const emm_grid *g, const emm_survey *s) {
  if (!g || !s) return EMM_EINVAL;
  if (!(s->omega0 > 0) || !(s->fmax > 0) || !(s->sigma_min > 0) || !std::isfinite(s->sigma_min)) return EMM_EINVAL;
  if (s->nt < 0 || s->nfreq < 1 || !s->freqs || s->nrec < 0 || (s->nrec > 0 && !s->rec)) return EMM_EINVAL;
  for (int f = 0; f < s->nfreq; ++f)
    if (!(s->freqs[f] > 0) || !std::isfinite(s->freqs[f])) return EMM_EINVAL;
  if (!std::isfinite(s->moment) || !std::isfinite(s->src_az) || !std::isfinite(s->src_dip)) return EMM_EINVAL;
  if (s->src_kind != 0 && s->src_kind != 1) return EMM_EINVAL;
  if (!(s->src_length >= 0) || !std::isfinite(s->src_length) ||
      (s->src_length > 0 && (s->src_points < 1 || s->src_points > 256)))
    return EMM_EINVAL;
  if (s->airwave != 0 && s->airwave != 1) return EMM_EINVAL;
  if (s->tile_shape != 0 && s->tile_shape != 1) return EMM_EINVAL;
  return EMM_OK;
}

// 4-D FP32 tensor [nsrc][np2][np1][pitch] (dims np0 x np1 x np2 x nsrc, the
// transmitters' state blocks sstride floats apart), box bx x by x bz x 1.
bool make_map(CUtensorMap *map, const float *base, const DevParams &p, int bx, int by, int bz) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {static_cast<cuuint64_t>(p.np[0]), static_cast<cuuint64_t>(p.np[1]),
                              static_cast<cuuint64_t>(p.np[2]), static_cast<cuuint64_t>(p.nsrc)};
  const cuuint64_t strides[3] = {static_cast<cuuint64_t>(p.pitch) * 4, static_cast<cuuint64_t>(p.plane) * 4,
                                 static_cast<cuuint64_t>(p.sstride) * 4};
  const cuuint32_t box[4] = {static_cast<cuuint32_t>(bx), static_cast<cuuint32_t>(by),
                             static_cast<cuuint32_t>(bz), 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The boxes of the three source fields (see Tiles).
template <int R, int S = 0>
bool make_tiles(TmaSet *t, float *const *F, const DevParams &p) {
  using T = Tiles<R, S>;
  return make_map(&t->m[0], F[0], p, TX, T::YH, T::ZQ) && make_map(&t->m[1], F[1], p, WX, T::TY, T::ZQ) &&
         make_map(&t->m[2], F[2], p, WX, T::YH, T::ZC);
}

// The four air transform passes after a half step (see k_air_fft).
template <bool MULTI, int KIND>
cudaError_t air_step(const DevParams &p, cudaStream_t st) {
  const int rd = p.air_rd, N0 = p.np[0], N1 = p.np[1];
  const int nin = KIND == 0 ? 2 : 1, nout = KIND == 0 ? 2 * (rd - 1) : 2 * rd;
  const unsigned z = static_cast<unsigned>(p.nsrc);
  const dim3 tb(AFT);
  const size_t s0 = 3 * sizeof(float2) * N0, s1 = 3 * sizeof(float2) * N1;
  cudaError_t e = cudaSuccess;
  if (std::max(s0, s1) > 48 * 1024) {  // lines of more than 2048 samples
    const int mx = static_cast<int>(std::max(s0, s1));
    e = cudaFuncSetAttribute(k_air_fft<0, MULTI, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_air_fft<1, MULTI, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_air_fft<2, MULTI, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_air_fft<3, MULTI, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return e;
  }
  e = launch_dependent(k_air_fft<0, MULTI, KIND>, dim3(nin * N1, 1, z), tb, s0, st, p);
  if (e == cudaSuccess) e = launch_dependent(k_air_fft<1, MULTI, KIND>, dim3(nin * N0, 1, z), tb, s1, st, p);
  if (e == cudaSuccess) e = launch_dependent(k_air_fft<2, MULTI, KIND>, dim3(nout * N0, 1, z), tb, s1, st, p);
  if (e == cudaSuccess) e = launch_dependent(k_air_fft<3, MULTI, KIND>, dim3(nout * N1, 1, z), tb, s0, st, p);
  return e;
}

// The second stream of split air runs and its events, one set per host
// thread and device, created on first use and kept for the life of the
// thread (a CUDA-graph capture may hold them).
struct AirSplitStreams {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, et = nullptr, eb = nullptr, ht = nullptr, hb = nullptr;
};

inline cudaError_t air_split_streams(AirSplitStreams **out) {
  constexpr int kDevs = 64;
  thread_local AirSplitStreams sets[kDevs];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
  AirSplitStreams &s = sets[dev];
  if (!s.side) {
    // the greatest priority: its CTAs (the critical path) are dispatched
    // ahead of the bulk launch's queued CTAs as SM slots free up
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s.side, cudaStreamNonBlocking, greatest);
    cudaEvent_t *ev[6] = {&s.fork, &s.join, &s.et, &s.eb, &s.ht, &s.hb};
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  *out = &s;
  return cudaSuccess;
}

// Air runs of an electric point dipole without the volume DTFT: each
// half-step is launched in two parts, the z-layers of tiles next to the air
// interface ("top": every cell above ks + R, with the receiver CTAs) and the
// rest ("bulk"), and the top part with the air transforms runs on a second
// stream beside the bulk part:
//   side:   E_top(n) -> air_E(n) -> H_top(n) -> air_H(n) -> E_top(n+1) ...
//   stream: E_bulk(n) -> H_bulk(n) -> E_bulk(n+1) ...
// with E_top(n) after H_bulk(n-1), E_bulk(n) after H_top(n-1), H_top(n)
// after E_bulk(n) and H_bulk(n) after E_top(n) (events).  Bulk cells lie at
// ks + R or deeper, so they never read the rows the air transforms write
// (rows above ks); the halo of each part is the other part's cells of the
// same time level, ordered by those events.  So the air transforms of a
// half-step overlap the bulk stencil launch of that half-step.  All launches
// are plain ones but the four air passes after a top launch, which follow
// it on the side stream as programmatic dependents.  Returns
// cudaErrorNotSupported (nothing enqueued) when the grid has no bulk layers.
template <int R, bool MULTI, int S>
cudaError_t launch_air_split(const DevParams &p, int n0, int n1, dim3 blocks, cudaStream_t st) {
  constexpr int ZC = shape_zc(S);
  const int lt = (p.air_ks + R - p.org[2] + ZC - 1) / ZC;  // top tile layers
  if (lt >= p.tiles_z) return cudaErrorNotSupported;
  DevParams qt = p, qb = p;
  qt.tiles_z = lt;  // the receiver layers and tile layers [0, lt)
  qb.rec_layers = 0;
  qb.tiles_z = p.tiles_z - lt;
  qb.org[2] = p.org[2] + lt * ZC;
  const dim3 gt(blocks.x, blocks.y, static_cast<unsigned>(p.rec_layers + lt));
  const dim3 gb(blocks.x, blocks.y, static_cast<unsigned>(p.tiles_z - lt));
  TmaSet tE{}, tH{};
  if (!make_tiles<R, S>(&tE, p.H, p) || !make_tiles<R, S>(&tH, p.E, p)) return cudaErrorInvalidValue;
  const size_t sb = smem_bytes<R, S>();
  cudaError_t e = cudaFuncSetAttribute(k_update_E<R, MULTI, false, false, S>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sb));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_H<R, MULTI, false, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sb));
  AirSplitStreams *ss = nullptr;
  if (e == cudaSuccess) e = air_split_streams(&ss);
  if (e != cudaSuccess) return e;
  PlainLaunches plain;
  cudaStream_t sd = ss->side;
  e = cudaEventRecord(ss->fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sd, ss->fork, 0);
  for (int n = n0; n < n1 && e == cudaSuccess; ++n) {
    // E half-step
    if (n > n0) e = cudaStreamWaitEvent(sd, ss->hb, 0);
    if (e == cudaSuccess) e = launch_dependent(k_update_E<R, MULTI, false, false, S>, gt, dim3(NT), sb, sd, qt, tE, n);
    if (e == cudaSuccess) e = cudaEventRecord(ss->et, sd);
    if (e == cudaSuccess && n > n0) e = cudaStreamWaitEvent(st, ss->ht, 0);
    if (e == cudaSuccess) e = launch_dependent(k_update_E<R, MULTI, false, false, S>, gb, dim3(NT), sb, st, qb, tE, n);
    if (e == cudaSuccess) e = cudaEventRecord(ss->eb, st);
    if (e == cudaSuccess && R > 1) {
      DependentLaunches chain;  // the four passes follow E_top on the side stream
      e = air_step<MULTI, 0>(p, sd);
    }
    // H half-step
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sd, ss->eb, 0);
    if (e == cudaSuccess) e = launch_dependent(k_update_H<R, MULTI, false, S>, gt, dim3(NT), sb, sd, qt, tH, n);
    if (e == cudaSuccess) e = cudaEventRecord(ss->ht, sd);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ss->et, 0);
    if (e == cudaSuccess) e = launch_dependent(k_update_H<R, MULTI, false, S>, gb, dim3(NT), sb, st, qb, tH, n);
    if (e == cudaSuccess) e = cudaEventRecord(ss->hb, st);
    if (e == cudaSuccess) {
      DependentLaunches chain;  // the four passes follow H_top on the side stream
      e = air_step<MULTI, 1>(p, sd);
    }
  }
  // join: the work after the run on `stream` waits for the side stream
  cudaError_t j = cudaEventRecord(ss->join, sd);
  if (j == cudaSuccess) j = cudaStreamWaitEvent(st, ss->join, 0);
  if (e == cudaSuccess) e = j;
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// OUT: one step whose E^{n+1} goes to p.Eout; the launches after the E
// half-step see it there.
template <int R, bool MULTI, bool CONV, bool OUT = false, int S = 0>
cudaError_t launch_steps(const DevParams &p, int n0, int n1, dim3 blocks, cudaStream_t st, StepEvents *te) {
  if (!OUT && !CONV && p.air_on && p.src_fused && !p.vacc && !te && n1 > n0) {
    const cudaError_t e = launch_air_split<R, MULTI, S>(p, n0, n1, blocks, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (OUT && (MULTI || CONV || n1 - n0 != 1)) return cudaErrorInvalidValue;
  DevParams q = p;
  q.ring_k = 1;  // the fields stay in place
  if (OUT)
    for (int a = 0; a < 3; ++a) q.E[a] = p.Eout[a];
  TmaSet tE{}, tH{};
  if (!make_tiles<R, S>(&tE, p.H, p) || !make_tiles<R, S>(&tH, q.E, p)) return cudaErrorInvalidValue;
  const size_t sb = smem_bytes<R, S>();
  cudaError_t e =
      cudaFuncSetAttribute(k_update_E<R, MULTI, CONV, OUT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(sb));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_H<R, MULTI, CONV, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sb));
  if (e != cudaSuccess) return e;
  // each half-step is launched as a programmatic dependent of the one before
  const dim3 inj(static_cast<unsigned>((p.nsrc * p.jstride + 127) / 128));  // k_inject threads
  size_t used = 0;
  if (te && te->loop[0]) cudaEventRecord(te->loop[0], st);
  for (int n = n0; n < n1 && e == cudaSuccess; ++n) {
    const bool timed = te && te->every > 0 && (n % te->every) == 0 && used + 4 <= te->ev.size();
    if (timed) cudaEventRecord(te->ev[used], st);
    e = launch_dependent(k_update_E<R, MULTI, CONV, OUT, S>, blocks, dim3(NT), sb, st, p, tE, n);
    if (e == cudaSuccess && !p.src_fused && !p.src_magnetic)
      e = launch_dependent(k_inject<MULTI, 0>, inj, dim3(128), 0, st, q, n);
    if (e == cudaSuccess && p.air_on && R > 1) e = air_step<MULTI, 0>(q, st);
    if (timed) cudaEventRecord(te->ev[used + 1], st);
    if (e == cudaSuccess && p.vacc)
      e = launch_volume(q, n, 1, [&](int, int c) -> const float * { return c < 3 ? q.E[c] : q.H[c - 3]; }, st);
    if (timed) {
      cudaEventRecord(te->ev[used + 2], st);
      te->vsteps.push_back(p.vacc ? 1 : 0);
    }
    if (e == cudaSuccess) e = launch_dependent(k_update_H<R, MULTI, CONV, S>, blocks, dim3(NT), sb, st, q, tH, n);
    if (e == cudaSuccess && p.src_magnetic) e = launch_dependent(k_inject<MULTI, 1>, inj, dim3(128), 0, st, q, n);
    if (e == cudaSuccess && p.air_on) e = air_step<MULTI, 1>(q, st);
    if (timed) {
      cudaEventRecord(te->ev[used + 3], st);
      used += 4;
      te->used += 1;
    }
  }
  if (te && te->loop[1]) cudaEventRecord(te->loop[1], st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// A one-transmitter solve with the volume DTFT over a ring of k = p.ring_k
// field slots (slot m mod k holds E^m and H^{m+1/2}).  The E half-step of
// step n reads E^n and H^{n+1/2} in slot n mod k and writes E^{n+1} into
// slot (n+1) mod k; the H half-step reads H^{n+1/2} and E^{n+1} and writes
// H^{n+3/2} into slot (n+1) mod k.  After the E launch (and the source and
// air launches after it) of the last step of each batch of at most k steps,
// and of the run's last step, one k_volume_dft launch adds the batch's
// terms.  The batch's fields are all still in the ring then: the first
// launch to overwrite one of its slots (the H launch of the batch's last
// step, or the E launch after it) follows the DTFT launch in stream order.
template <int R, int S>
cudaError_t launch_ring(const DevParams &p, int n0, int n1, dim3 blocks, cudaStream_t st, StepEvents *te) {
  const int k = p.ring_k;
  if (k < 2 || k > kRing || !p.vacc || p.nsrc != 1 || p.corner || p.Eout[0]) return cudaErrorInvalidValue;
  auto slot = [&](int sl, int c) { return const_cast<float *>(ring_field(p, sl, c)); };
  // tensor maps per slot: the H boxes the E launch reads, the E boxes the H launch reads
  TmaSet tE[kRing], tH[kRing];
  for (int sl = 0; sl < k; ++sl) {
    float *Hs[3] = {slot(sl, 3), slot(sl, 4), slot(sl, 5)};
    float *Es[3] = {slot(sl, 0), slot(sl, 1), slot(sl, 2)};
    if (!make_tiles<R, S>(&tE[sl], Hs, p) || !make_tiles<R, S>(&tH[sl], Es, p)) return cudaErrorInvalidValue;
  }
  const size_t sb = smem_bytes<R, S>();
  cudaError_t e = cudaFuncSetAttribute(k_update_E<R, false, false, true, S>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sb));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_H<R, false, false, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sb));
  if (e != cudaSuccess) return e;
  const dim3 inj(static_cast<unsigned>((p.jstride + 127) / 128));  // k_inject threads
  // timed samples: the last step of every stride-th batch
  const int stride = te && te->every > 0 ? std::max(1, te->every / k) : 0;
  size_t used = 0;
  int batch = 0, b0 = n0;
  if (te && te->loop[0]) cudaEventRecord(te->loop[0], st);
  for (int n = n0; n < n1 && e == cudaSuccess; ++n) {
    const int so = n % k, sn = (n + 1) % k;
    const bool flush = n - b0 + 1 == k || n == n1 - 1;
    const bool timed = flush && stride > 0 && batch % stride == 0 && used + 4 <= te->ev.size();
    DevParams q = p;  // E half-step: E^n, H^{n+1/2} in slot so; E^{n+1} into slot sn
    for (int c = 0; c < 3; ++c) {
      q.E[c] = slot(so, c);
      q.H[c] = slot(so, 3 + c);
      q.Eout[c] = slot(sn, c);
    }
    if (timed) cudaEventRecord(te->ev[used], st);
    e = launch_dependent(k_update_E<R, false, false, true, S>, blocks, dim3(NT), sb, st, q, tE[so], n);
    for (int c = 0; c < 3; ++c) {  // the launches after it see E^{n+1}
      q.E[c] = slot(sn, c);
      q.Eout[c] = nullptr;
    }
    if (e == cudaSuccess && !p.src_fused && !p.src_magnetic)
      e = launch_dependent(k_inject<false, 0>, inj, dim3(128), 0, st, q, n);
    if (e == cudaSuccess && p.air_on && R > 1) e = air_step<false, 0>(q, st);
    if (timed) cudaEventRecord(te->ev[used + 1], st);
    if (e == cudaSuccess && flush) {
      e = launch_volume(p, b0, n - b0 + 1, [&](int m, int c) -> const float * {
        return c < 3 ? slot((m + 1) % k, c) : slot(m % k, c);  // E^{m+1}, H^{m+1/2}
      }, st);
      if (timed) te->vsteps.push_back(n - b0 + 1);
      b0 = n + 1;
      ++batch;
    }
    if (timed) cudaEventRecord(te->ev[used + 2], st);
    for (int c = 0; c < 3; ++c) q.Hout[c] = slot(sn, 3 + c);  // H^{n+3/2} into slot sn
    if (e == cudaSuccess) e = launch_dependent(k_update_H<R, false, false, S, true>, blocks, dim3(NT), sb, st, q, tH[sn], n);
    for (int c = 0; c < 3; ++c) {
      q.H[c] = slot(sn, 3 + c);
      q.Hout[c] = nullptr;
    }
    if (e == cudaSuccess && p.src_magnetic) e = launch_dependent(k_inject<false, 1>, inj, dim3(128), 0, st, q, n);
    if (e == cudaSuccess && p.air_on) e = air_step<false, 1>(q, st);
    if (timed) {
      cudaEventRecord(te->ev[used + 3], st);
      used += 4;
      te->used += 1;
    }
  }
  if (te && te->loop[1]) cudaEventRecord(te->loop[1], st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// Normalisation of the DTFT (Eq. 7) for a run of nsteps leapfrog steps, as
// complex pairs [2][nfreq][2] for the E and the H components.  Electric
// source: sqrt(-i w / (2 w0)) / J'(f) and 1 / J'(f), J' the DTFT of the
// wavelet sampled at t_{n+1/2}; magnetic source: 1 / M'(f) and
// 1 / (sqrt(-i w / (2 w0)) M'(f)), M' sampled at t_{n+1}.
void normalisation(const emm_survey *s, double dt, int nsteps, double *norm) {
  const int nf = s->nfreq;
  const std::complex<double> I(0.0, 1.0);
  const double t0 = 1.5 / s->fmax;
  for (int f = 0; f < nf; ++f) {
    const std::complex<double> wp = std::complex<double>(1.0, 1.0) * std::sqrt(2.0 * M_PI * s->freqs[f] * s->omega0);
    std::complex<double> jhat = 0.0;
    for (int n = 0; n < nsteps; ++n) {
      const double ts = (n + (s->src_kind == 1 ? 1.0 : 0.5)) * dt;
      const double u = M_PI * s->fmax * (ts - t0);
      const double a = s->moment * std::exp(-u * u);
      jhat += std::exp(I * wp * ts) * dt * a;
    }
    const std::complex<double> sE =
        std::sqrt(2.0 * M_PI * s->freqs[f] / (2.0 * s->omega0)) * std::exp(-I * (M_PI / 4.0));
    // electric source: G^EE = sE E'/J', G^HE = H'/J'; magnetic: G^EH = E'/M',
    // G^HH = H'/(sE M')
    const bool mag = s->src_kind == 1;
    const std::complex<double> nE = (jhat != 0.0) ? (mag ? 1.0 / jhat : sE / jhat) : 0.0;
    const std::complex<double> nH = (jhat != 0.0) ? (mag ? 1.0 / (sE * jhat) : 1.0 / jhat) : 0.0;
    norm[2 * f] = nE.real();
    norm[2 * f + 1] = nE.imag();
    norm[2 * nf + 2 * f] = nH.real();
    norm[2 * nf + 2 * f + 1] = nH.imag();
  }
}

int prepare_forward(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                    double *rec_out, double *vol_out, cudaStream_t cs, Prepared *out, int nsrc,
                    const double *src_pos, bool converge, bool upload_tables, int shape) {
  int st = check_survey(g, s);
  if (st != EMM_OK) return st;
  if (!sigma || !ws || (s->nrec > 0 && !rec_out) || (s->volume && !vol_out)) return EMM_EINVAL;
  if (nsrc < 1 || (nsrc > 1 && s->volume)) return EMM_EINVAL;
  const Layout L = plan(g, s, nsrc);
  if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return EMM_EWORKSPACE;
  const int rd = g->rd, m = 2 * rd, nf = s->nfreq, nt = s->nt, nb = g->nb;
  const int nbe = g->nb + g->ne;

  // time step (Sec. 3.2) and vmax
  double dt_max, eta, vmax;
  st = emm_time_step(g, s->sigma_min, s->omega0, &dt_max, &eta, &vmax);
  if (st != EMM_OK) return st;
  const double dt = (s->dt > 0) ? s->dt : dt_max;
  if (dt * eta > 1.0) return EMM_ECFL;

  // ---- host tables, packed at their workspace offsets ----
  const size_t tab0 = L.cm[0];
  std::vector<unsigned char> blob;
  try {
    blob.assign(L.total - tab0, 0);
  } catch (const std::bad_alloc &) {
    return EMM_ENOMEM;
  }
  auto at = [&](size_t off) { return blob.data() + (off - tab0); };
  for (int a = 0; a < 3; ++a) {
    const Axis &ax = g->ax[a];
    float *cm = reinterpret_cast<float *>(at(L.cm[a]));
    float *cp = reinterpret_cast<float *>(at(L.cp[a]));
    for (size_t q = 0; q < ax.cm.size(); ++q) cm[q] = static_cast<float>(ax.cm[q]);
    for (size_t q = 0; q < ax.cp.size(); ++q) cp[q] = static_cast<float>(ax.cp[q]);
    std::vector<double> ab(8 * static_cast<size_t>(nb));
    cpml_axis(g, a, vmax, s->fmax, dt, ab.data());
    // air above the model: no CPML on the top face (a = b = 0 on the near z slab)
    if (s->airwave && a == 2)
      for (int grp = 0; grp < 4; ++grp)
        for (int e = 0; e < nb; ++e) ab[static_cast<size_t>(grp) * 2 * nb + e] = 0.0;
    float *pm = reinterpret_cast<float *>(at(L.pml[a]));
    for (size_t q = 0; q < ab.size(); ++q) pm[q] = static_cast<float>(ab[q]);
  }
  // sources: J_node = moment s(t) dir_c w_node / V_node, V = dual-cell volume,
  // one stencil set per transmitter
  const double dir[3] = {std::cos(s->src_dip) * std::cos(s->src_az), std::cos(s->src_dip) * std::sin(s->src_az),
                         std::sin(s->src_dip)};
  DevParams p{};
  SrcDev *srcs = reinterpret_cast<SrcDev *>(at(L.srcs));
  for (int k = 0; k < nsrc; ++k) {
    const double *pos = src_pos ? src_pos + 3 * k : s->src;
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(pos[a])) return EMM_EINVAL;
    SrcDev &sd = srcs[k];
    sd = SrcDev{};
    for (int a = 0; a < 3; ++a) {
      sd.lo[a] = 1 << 30;
      sd.hi[a] = -1;
    }
    // the stencils sit on the E samples of an electric dipole, on the H
    // samples of a magnetic one; an antenna is npt sub-dipoles at the
    // midpoints of equal segments along dir, each with 1/npt of the moment,
    // whose weights are summed on the union of their boxes
    const int sc = s->src_kind == 1 ? 3 : 0;
    const int npt = s->src_length > 0 ? s->src_points : 1;
    int ext[3];
    source_box_bound(g, s, ext);
    const size_t jstride = source_stride(g, s), cv = jstride / 3;
    for (int c = 0; c < 3; ++c) {
      if (dir[c] == 0.0) continue;
      std::vector<int> starts(static_cast<size_t>(npt) * 3);
      std::vector<double> ws(static_cast<size_t>(npt) * 3 * m);
      int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
      for (int q = 0; q < npt; ++q) {
        const double off = s->src_length > 0 ? (-0.5 + (q + 0.5) / npt) * s->src_length : 0.0;
        for (int a = 0; a < 3; ++a) {
          const double pa = pos[a] + off * dir[a];
          st = locate_axis(g, a, kHalf[c + sc][a], pa, &starts[q * 3 + a], &ws[(static_cast<size_t>(q) * 3 + a) * m]);
          if (st != EMM_OK) return st;
          // with air above the model the source stencil stays below the interface
          if (s->airwave && a == 2 && starts[q * 3 + 2] < nbe) return EMM_EOUTSIDE;
          lo[a] = std::min(lo[a], starts[q * 3 + a]);
          hi[a] = std::max(hi[a], starts[q * 3 + a] + m - 1);
        }
      }
      int box[3];
      for (int a = 0; a < 3; ++a) {
        box[a] = hi[a] - lo[a] + 1;
        if (box[a] > ext[a]) return EMM_EINVAL;
      }
      std::vector<double> acc(static_cast<size_t>(box[0]) * box[1] * box[2], 0.0);
      for (int q = 0; q < npt; ++q)
        for (int q3 = 0; q3 < m; ++q3)
          for (int q2 = 0; q2 < m; ++q2)
            for (int q1 = 0; q1 < m; ++q1) {
              const int idx[3] = {starts[q * 3] + q1, starts[q * 3 + 1] + q2, starts[q * 3 + 2] + q3};
              double vol = 1.0;
              for (int a = 0; a < 3; ++a) {
                const Axis &ax = g->ax[a];
                vol *= kHalf[c + sc][a] ? (ax.X[idx[a] + 1] - ax.X[idx[a]]) : (ax.Xh[idx[a]] - ax.Xh[idx[a] - 1]);
              }
              const double *w = &ws[static_cast<size_t>(q) * 3 * m];
              acc[(static_cast<size_t>(idx[2] - lo[2]) * box[1] + (idx[1] - lo[1])) * box[0] + (idx[0] - lo[0])] +=
                  dir[c] * w[q1] * w[m + q2] * w[2 * m + q3] / vol / npt;
            }
      float *jw = reinterpret_cast<float *>(at(L.jw)) + static_cast<size_t>(k) * jstride + c * cv;
      for (size_t q = 0; q < acc.size(); ++q) jw[q] = static_cast<float>(acc[q]);
      sd.on[c] = 1;
      sd.any = 1;
      sd.woff[c] = static_cast<int>(c * cv);
      for (int a = 0; a < 3; ++a) {
        sd.start[c][a] = lo[a];
        sd.box[c][a] = box[a];
        sd.lo[a] = std::min(sd.lo[a], lo[a]);
        sd.hi[a] = std::max(sd.hi[a], hi[a]);
      }
    }
  }
  // receivers: stencils of all six components
  int *rs = reinterpret_cast<int *>(at(L.rec_start));
  double *rw = reinterpret_cast<double *>(at(L.rec_w));
  for (int r = 0; r < s->nrec; ++r)
    for (int c = 0; c < 6; ++c)
      for (int a = 0; a < 3; ++a) {
        st = locate_axis(g, a, kHalf[c][a], s->rec[3 * r + a], &rs[(r * 6 + c) * 3 + a],
                         rw + (static_cast<size_t>(r * 6 + c) * 3 + a) * m);
        if (st != EMM_OK) return st;
      }
  // wavelet samples at t_{n+1/2} and DTFT factors e^{i w' t} dt, w' = (1+i) sqrt(w w0)
  float *amp = reinterpret_cast<float *>(at(L.amp));
  double *fE = reinterpret_cast<double *>(at(L.fE)), *fH = reinterpret_cast<double *>(at(L.fH));
  float *fE32 = reinterpret_cast<float *>(at(L.fE32)), *fH32 = reinterpret_cast<float *>(at(L.fH32));
  std::vector<std::complex<double>> wp(nf);
  for (int f = 0; f < nf; ++f)
    wp[f] = std::complex<double>(1.0, 1.0) * std::sqrt(2.0 * M_PI * s->freqs[f] * s->omega0);
  const double t0 = 1.5 / s->fmax;
  const std::complex<double> I(0.0, 1.0);
  for (int n = 0; n < nt; ++n) {
    const double th = (n + 0.5) * dt, te_ = (n + 1.0) * dt;
    // J is sampled at t_{n+1/2} (the E update's centre), M at t_{n+1} (the H update's)
    const double u = M_PI * s->fmax * ((s->src_kind == 1 ? te_ : th) - t0);
    const double a = s->moment * std::exp(-u * u);
    amp[n] = static_cast<float>(a);
    for (int f = 0; f < nf; ++f) {
      const std::complex<double> eE = std::exp(I * wp[f] * te_) * dt, eH = std::exp(I * wp[f] * th) * dt;
      const size_t o = (static_cast<size_t>(n) * nf + f) * 2;
      fE[o] = eE.real();
      fE[o + 1] = eE.imag();
      fH[o] = eH.real();
      fH[o + 1] = eH.imag();
      fE32[o] = static_cast<float>(eE.real());
      fE32[o + 1] = static_cast<float>(eE.imag());
      fH32[o] = static_cast<float>(eH.real());
      fH32[o + 1] = static_cast<float>(eH.imag());
    }
  }
  normalisation(s, dt, nt, reinterpret_cast<double *>(at(L.norm)));

  // air above the model (Sec. 3.3): DFT twiddles e^{-2 pi i m / N} and the
  // continuation factors, per horizontal wavenumber k (kx = 2 pi p / (N dx),
  // p in (-N/2, N/2]): e^{-|k| h} for the E rows at the heights h above the
  // interface, and i k_{x,y} / |k| e^{-i k_{x,y} d_{x,y} / 2} e^{-|k| h} for the
  // H_x, H_y half rows (0 at k = 0)
  if (s->airwave) {
    const int N0 = g->ax[0].npad, N1 = g->ax[1].npad, ks = nbe;
    double d[2];
    for (int a = 0; a < 2; ++a) {
      const Axis &ax = g->ax[a];
      d[a] = ax.X[1] - ax.X[0];
      for (size_t i = 1; i < ax.X.size(); ++i)
        if (std::fabs((ax.X[i] - ax.X[i - 1]) - d[a]) > 1e-9 * d[a]) return EMM_EINVAL;
    }
    float2 *twx = reinterpret_cast<float2 *>(at(L.air_twx)), *twy = reinterpret_cast<float2 *>(at(L.air_twy));
    // the roots of unity W[m] = e^{-2 pi i m / N}
    for (int m = 0; m < N0; ++m)
      twx[m] = make_float2(static_cast<float>(std::cos(2 * M_PI * m / N0)), static_cast<float>(-std::sin(2 * M_PI * m / N0)));
    for (int m = 0; m < N1; ++m)
      twy[m] = make_float2(static_cast<float>(std::cos(2 * M_PI * m / N1)), static_cast<float>(-std::sin(2 * M_PI * m / N1)));
    const Axis &az = g->ax[2];
    float *decE = reinterpret_cast<float *>(at(L.air_decE));
    float2 *facH = reinterpret_cast<float2 *>(at(L.air_facH));
    const size_t plane2 = static_cast<size_t>(N0) * N1;
    for (int k = 0; k < N1; ++k)
      for (int q = 0; q < N0; ++q) {
        const double kx = 2 * M_PI * (q <= N0 / 2 ? q : q - N0) / (N0 * d[0]);
        const double ky = 2 * M_PI * (k <= N1 / 2 ? k : k - N1) / (N1 * d[1]);
        const double kk = std::sqrt(kx * kx + ky * ky);
        const size_t o = static_cast<size_t>(k) * N0 + q;
        for (int r = 0; r + 1 < rd; ++r) decE[r * plane2 + o] = static_cast<float>(std::exp(-kk * (az.X[ks] - az.X[ks - 1 - r])));
        for (int r = 0; r < rd; ++r) {
          const double decay = std::exp(-kk * (az.X[ks] - az.Xh[ks - 1 - r]));
          for (int dd = 0; dd < 2; ++dd) {
            const double kd = dd == 0 ? kx : ky;
            const std::complex<double> f =
                kk > 0 ? I * (kd / kk) * std::exp(-I * (kd * d[dd] / 2)) * decay : std::complex<double>(0.0);
            facH[(static_cast<size_t>(dd) * rd + r) * plane2 + o] =
                make_float2(static_cast<float>(f.real()), static_cast<float>(f.imag()));
          }
        }
      }
  }

  // ---- device parameters ----
  unsigned char *base = static_cast<unsigned char *>(ws);
  for (int a = 0; a < 3; ++a) {
    p.np[a] = g->ax[a].npad;
    p.n[a] = g->ax[a].n;
    p.cm[a] = reinterpret_cast<const float *>(base + L.cm[a]);
    p.cp[a] = reinterpret_cast<const float *>(base + L.cp[a]);
    p.pml[a] = reinterpret_cast<const float *>(base + L.pml[a]);
  }
  if (shape < 0) shape = converge ? 0 : s->tile_shape;  // convergence runs keep the 32 x 8 x 2 tiles
  if (shape < 0 || shape >= kShapes) return EMM_EINVAL;
  const FieldGeom fg = field_geom(g, shape);
  p.pitch = fg.pitch;
  p.plane = static_cast<size_t>(p.pitch) * p.np[1];
  p.nbe = nbe;
  p.nb = nb;
  for (int c = 0; c < 3; ++c) {
    p.E[c] = reinterpret_cast<float *>(base + L.E[c]) + fg.xshift;
    p.H[c] = reinterpret_cast<float *>(base + L.H[c]) + fg.xshift;
    p.ie[c] = reinterpret_cast<const float *>(base + L.ie[c]) + fg.xshift;
  }
  // a convergence run keeps its fields in place (its stop step is decided on
  // the device, so the DTFT of every step must follow that step)
  p.ring_k = converge ? 1 : L.ring_k;
  p.ring = reinterpret_cast<float *>(base + L.ring) + fg.xshift;
  p.ring_comp = L.ring_comp / 4;
  for (int c = 0; c < 6; ++c) {
    // y- and z-derivative arrays share the field rows' x shift
    const int shift = psi_axis(c) == 0 ? 0 : fg.xshift;
    p.psiE[c] = reinterpret_cast<float *>(base + L.psiE[c]) + shift;
    p.psiH[c] = reinterpret_cast<float *>(base + L.psiH[c]) + shift;
  }
  for (int h = 0; h < 2; ++h) {
    p.psx_hx[h] = fg.psx_hx[h];
    p.psx_wx[h] = fg.psx_wx[h];
    p.psx_far0[h] = fg.psx_far0[h];
  }
  p.nsrc = nsrc;
  p.sstride = L.sstride / 4;
  p.srcs = reinterpret_cast<const SrcDev *>(base + L.srcs);
  p.jw = reinterpret_cast<const float *>(base + L.jw);
  p.dt_mu = static_cast<float>(dt / kMu0);
  p.amp = reinterpret_cast<const float *>(base + L.amp);
  p.nrec = s->nrec;
  p.nf = nf;
  p.rec_start = reinterpret_cast<const int *>(base + L.rec_start);
  p.rec_w = reinterpret_cast<const double *>(base + L.rec_w);
  p.rec_acc = rec_out;
  p.fE = reinterpret_cast<const double *>(base + L.fE);
  p.fH = reinterpret_cast<const double *>(base + L.fH);
  p.fE32 = reinterpret_cast<const float *>(base + L.fE32);
  p.fH32 = reinterpret_cast<const float *>(base + L.fH32);
  p.vacc = s->volume ? reinterpret_cast<float4 *>(base + L.vacc) : nullptr;
  p.status = reinterpret_cast<int *>(base + L.status);
  p.src_magnetic = s->src_kind == 1 ? 1 : 0;
  p.src_fused = (s->src_kind == 0 && !(s->src_length > 0)) ? 1 : 0;
  if (s->airwave) {
    p.air_on = 1;
    p.air_ks = nbe;
    p.air_rd = rd;
    p.air_twx = reinterpret_cast<const float2 *>(base + L.air_twx);
    p.air_twy = reinterpret_cast<const float2 *>(base + L.air_twy);
    p.air_decE = reinterpret_cast<const float *>(base + L.air_decE);
    p.air_facH = reinterpret_cast<const float2 *>(base + L.air_facH);
    const size_t plane2 = static_cast<size_t>(p.np[0]) * p.np[1];
    p.air_T = reinterpret_cast<float2 *>(base + L.air_work);
    p.air_F = p.air_T + static_cast<size_t>(nsrc) * 3 * plane2;
    p.air_U = p.air_F + static_cast<size_t>(nsrc) * 3 * plane2;
  }
  p.jstride = source_stride(g, s);
  if (converge) {
    p.corner = reinterpret_cast<double *>(base + L.conv);
    p.halt = reinterpret_cast<const int *>(base + L.conv + 2 * 8 * 6 * 2 * sizeof(double));
    p.conv_f = 0;
    for (int f = 1; f < nf; ++f)
      if (s->freqs[f] < s->freqs[p.conv_f]) p.conv_f = f;
  }
  // launch shape: TX x TY column tiles times runs of ZC planes, then the
  // receiver CTAs (one warp per receiver component)
  for (int a = 0; a < 3; ++a) p.org[a] = fg.org[a];
  p.tiles_x = fg.tiles[0];
  p.tiles_y = fg.tiles[1];
  p.tiles_z = fg.tiles[2];
  int sms = 148;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  p.stencil_blocks = p.tiles_x * p.tiles_y * p.tiles_z;
  p.rec_blocks = (s->nrec * 3 + (converge ? 1 : 0) + NT / 32 - 1) / (NT / 32);
  const int layer = p.tiles_x * p.tiles_y;
  p.rec_layers = (p.rec_blocks + layer - 1) / layer;
  const dim3 blocks(p.tiles_x * nsrc, p.tiles_y, p.rec_layers + p.tiles_z);

  // ---- enqueue ----
  cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_end, cs);
  if (e == cudaSuccess && s->nrec > 0)
    e = cudaMemsetAsync(rec_out, 0, static_cast<size_t>(nsrc) * s->nrec * 6 * nf * 2 * sizeof(double), cs);
  if (e == cudaSuccess && upload_tables)
    e = cudaMemcpyAsync(base + tab0, blob.data(), blob.size(), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return EMM_ECUDA;
  k_prepare<<<4 * sms, 256, 0, cs>>>(sigma, reinterpret_cast<float *>(base + L.ie[0]),
                                     reinterpret_cast<float *>(base + L.ie[1]),
                                     reinterpret_cast<float *>(base + L.ie[2]), p.n[0], p.n[1], p.n[2], p.np[0],
                                     p.np[1], p.np[2], p.pitch, fg.xshift, nbe, 2.0 * s->omega0 * dt, s->sigma_min,
                                     p.status);
  out->p = p;
  out->L = L;
  out->fg = fg;
  out->blocks = blocks;
  out->dt = dt;
  out->sms = sms;
  out->rd = rd;
  out->shape = shape;
  return cudaGetLastError() == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

// The launch variants of one order: one transmitter; a batch; a convergence
// run; one step into another E buffer.
template <int R, int S>
cudaError_t run_order(const DevParams &p, dim3 blocks, int n0, int n1, cudaStream_t cs, StepEvents *te) {
  // the gradient's one-step runs and convergence runs use the 32 x 8 x 2 tiles
  if (p.Eout[0]) return S == 0 ? launch_steps<R, false, false, true>(p, n0, n1, blocks, cs, te) : cudaErrorInvalidValue;
  if (p.nsrc > 1) return launch_steps<R, true, false, false, S>(p, n0, n1, blocks, cs, te);
  if (p.corner) return S == 0 ? launch_steps<R, false, true>(p, n0, n1, blocks, cs, te) : cudaErrorInvalidValue;
  if (p.ring_k > 1) return launch_ring<R, S>(p, n0, n1, blocks, cs, te);
  return launch_steps<R, false, false, false, S>(p, n0, n1, blocks, cs, te);
}

cudaError_t run_steps(const Prepared &P, const DevParams &p, dim3 blocks, int n0, int n1, cudaStream_t cs,
                      StepEvents *te) {
  switch (2 * P.rd + P.shape) {
    case 2: return run_order<1, 0>(p, blocks, n0, n1, cs, te);
    case 3: return run_order<1, 1>(p, blocks, n0, n1, cs, te);
    case 4: return run_order<2, 0>(p, blocks, n0, n1, cs, te);
    case 5: return run_order<2, 1>(p, blocks, n0, n1, cs, te);
    case 6: return run_order<3, 0>(p, blocks, n0, n1, cs, te);
    case 7: return run_order<3, 1>(p, blocks, n0, n1, cs, te);
    case 8: return run_order<4, 0>(p, blocks, n0, n1, cs, te);
    default: return run_order<4, 1>(p, blocks, n0, n1, cs, te);
  }
}

// Work-list solve of prepared problems P (one order R): every leapfrog step
// is one E and one H launch over all of them.
template <int R>
cudaError_t launch_jobs(const std::vector<Prepared> &P, const std::vector<int> &nts, cudaStream_t st) {
  const int nj = static_cast<int>(P.size());
  std::unique_ptr<JobSet> JE(new JobSet{}), JH(new JobSet{});
  int total = 0, nmax = 0;
  for (int j = 0; j < nj; ++j) {
    const DevParams &p = P[j].p;
    if (!make_tiles<R>(&JE->tm[j], p.H, p) || !make_tiles<R>(&JH->tm[j], p.E, p)) return cudaErrorInvalidValue;
    JE->p[j] = JH->p[j] = p;
    JE->cta0[j] = JH->cta0[j] = total;
    JE->nt[j] = JH->nt[j] = nts[j];
    total += static_cast<int>(P[j].blocks.x * P[j].blocks.y * P[j].blocks.z);
    nmax = std::max(nmax, nts[j]);
  }
  JE->cta0[nj] = JH->cta0[nj] = total;
  JE->njobs = JH->njobs = nj;
  const size_t sb = smem_bytes<R>();
  cudaError_t e = cudaFuncSetAttribute(k_update_E_jobs<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sb));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_H_jobs<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sb));
  for (int n = 0; n < nmax && e == cudaSuccess; ++n) {
    e = launch_dependent(k_update_E_jobs<R>, dim3(static_cast<unsigned>(total)), dim3(NT), sb, st, *JE, n);
    if (e == cudaSuccess)
      e = launch_dependent(k_update_H_jobs<R>, dim3(static_cast<unsigned>(total)), dim3(NT), sb, st, *JH, n);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// Workspace slices of a work list: each problem's forward workspace, 256-byte
// aligned, one after the other.
int jobs_layout(int nj, const emm_job *jobs, std::vector<size_t> *off, size_t *total) {
  if (nj < 1 || nj > kMaxJobs || !jobs) return EMM_EINVAL;
  size_t o = 0;
  off->clear();
  for (int j = 0; j < nj; ++j) {
    const emm_survey *s = jobs[j].survey;
    const int st = check_survey(jobs[j].grid, s);
    if (st != EMM_OK) return st;
    if (s->volume || s->airwave || s->src_kind != 0 || s->src_length > 0 || jobs[j].grid->rd != jobs[0].grid->rd)
      return EMM_EINVAL;
    off->push_back(o);
    o = align_up(o + plan(jobs[j].grid, s).total);
  }
  *total = o;
  return EMM_OK;
}

// Steps n0 .. n1-1 of prepared problems by one strategy (EMM_JOBS_*): the
// work-list launches; each problem's steps in turn on cs; or each problem on
// a stream of its own, forked from cs and joined back to it.
cudaError_t run_jobs(const std::vector<Prepared> &P, const std::vector<int> &nts, int strategy, int n0, int n1,
                     cudaStream_t cs) {
  const int nj = static_cast<int>(P.size());
  std::vector<int> ends(nj);
  for (int j = 0; j < nj; ++j) ends[j] = std::min(nts[j], n1);
  if (strategy == EMM_JOBS_LIST) {
    if (n0 != 0) return cudaErrorInvalidValue;
    switch (P[0].rd) {
      case 1: return launch_jobs<1>(P, ends, cs);
      case 2: return launch_jobs<2>(P, ends, cs);
      case 3: return launch_jobs<3>(P, ends, cs);
      default: return launch_jobs<4>(P, ends, cs);
    }
  }
  if (strategy == EMM_JOBS_SEQUENTIAL) {
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < nj && e == cudaSuccess; ++j)
      if (n0 < ends[j]) e = run_steps(P[j], P[j].p, P[j].blocks, n0, ends[j], cs, nullptr);
    return e;
  }
  // EMM_JOBS_STREAMS: the streams and events are released once their work is
  // done.  The problems' launches on these streams are plain ones, not
  // programmatic dependents: after a CUDA-graph plan had run in the process,
  // dependent-launch chains on several such streams at once were seen never
  // to finish on the eight uneven grids.
  PlainLaunches plain;
  cudaEvent_t fork;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(fork, cs);
  for (int j = 0; j < nj && e == cudaSuccess; ++j) {
    cudaStream_t sj;
    cudaEvent_t done;
    e = cudaStreamCreateWithFlags(&sj, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sj, fork, 0);
    if (e == cudaSuccess && n0 < ends[j]) e = run_steps(P[j], P[j].p, P[j].blocks, n0, ends[j], sj, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(done, sj);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, done, 0);
    cudaEventDestroy(done);
    cudaStreamDestroy(sj);
  }
  cudaEventDestroy(fork);
  return e;
}

int prepare_jobs(int nj, const emm_job *jobs, void *ws, size_t ws_bytes, cudaStream_t cs, std::vector<Prepared> *P,
                 std::vector<int> *nts) {
  std::vector<size_t> off;
  size_t total = 0;
  int st = jobs_layout(nj, jobs, &off, &total);
  if (st != EMM_OK) return st;
  if (!ws || ws_bytes < total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return EMM_EWORKSPACE;
  for (int j = 0; j < nj; ++j)
    if (!jobs[j].sigma || (jobs[j].survey->nrec > 0 && !jobs[j].rec_out)) return EMM_EINVAL;
  unsigned char *base = static_cast<unsigned char *>(ws);
  P->assign(nj, Prepared{});
  nts->assign(nj, 0);
  for (int j = 0; j < nj; ++j) {
    const size_t end = j + 1 < nj ? off[j + 1] : total;
    st = prepare_forward(jobs[j].grid, jobs[j].survey, jobs[j].sigma, base + off[j], end - off[j], jobs[j].rec_out,
                         nullptr, cs, &(*P)[j], 1, nullptr, false, true, 0);
    if (st != EMM_OK) return st;
    (*nts)[j] = jobs[j].survey->nt;
  }
  return EMM_OK;
}

int forward_jobs_impl(int nj, const emm_job *jobs, int strategy, void *ws, size_t ws_bytes, cudaStream_t cs) {
  if (strategy < EMM_JOBS_LIST || strategy > EMM_JOBS_STREAMS) return EMM_EINVAL;
  std::vector<Prepared> P;
  std::vector<int> nts;
  int st = prepare_jobs(nj, jobs, ws, ws_bytes, cs, &P, &nts);
  if (st != EMM_OK) return st;
  const int nmax = *std::max_element(nts.begin(), nts.end());
  if (run_jobs(P, nts, strategy, 0, nmax, cs) != cudaSuccess) return EMM_ECUDA;
  for (int j = 0; j < nj; ++j) {
    st = finalize_forward(P[j], jobs[j].survey, jobs[j].rec_out, nullptr, cs);
    if (st != EMM_OK) return st;
  }
  return EMM_OK;
}

// Times the first `steps` leapfrog steps (at most each problem's own) of
// every strategy on the problems (after a warm-up of a few steps each) and
// returns the fastest.  Synchronises cs;
// leaves the workspace to be prepared again by the next solve.
int jobs_tune(int nj, const emm_job *jobs, void *ws, size_t ws_bytes, int steps, cudaStream_t cs, double *ms,
              int *best) {
  if (steps < 1 || !ms || !best) return EMM_EINVAL;
  std::vector<Prepared> P;
  std::vector<int> nts;
  int st = prepare_jobs(nj, jobs, ws, ws_bytes, cs, &P, &nts);
  if (st != EMM_OK) return st;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return EMM_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return EMM_ECUDA;
  }
  cudaError_t e = cudaSuccess;
  for (int k = EMM_JOBS_LIST; k <= EMM_JOBS_STREAMS && e == cudaSuccess; ++k) {
    e = run_jobs(P, nts, k, 0, std::min(steps, 4), cs);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, cs);
    if (e == cudaSuccess) e = run_jobs(P, nts, k, 0, steps, cs);
    if (e == cudaSuccess) e = cudaEventRecord(b, cs);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    ms[k] = t;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return EMM_ECUDA;
  *best = EMM_JOBS_LIST;
  for (int k = EMM_JOBS_LIST; k <= EMM_JOBS_STREAMS; ++k)
    if (ms[k] < ms[*best]) *best = k;
  return EMM_OK;
}

// ---- persistent work list (k_persist) ----
// Workspace: a 256-byte header (status word at 0, so emm_status(ws) reads
// the work list's status; abort word; arrival counter), then each task's
// forward workspace, 256-byte aligned.
constexpr size_t kPHdrStatus = 0, kPHdrAbort = 4, kPHdrBar = 8, kPHdrClaim = 16;

int persist_layout(int nt, const emm_task *t, std::vector<size_t> *off, size_t *total) {
  if (nt < 1 || nt > kMaxTasks || !t) return EMM_EINVAL;
  size_t o = kAlign;
  off->clear();
  for (int j = 0; j < nt; ++j) {
    const emm_survey *s = t[j].survey;
    const int st = check_survey(t[j].grid, s);
    if (st != EMM_OK) return st;
    if (s->volume || s->airwave || s->src_kind != 0 || s->src_length > 0 || t[j].grid->rd != t[0].grid->rd ||
        t[j].nsrc < 1 || (t[j].nsrc > 1 && !t[j].src_pos))
      return EMM_EINVAL;
    off->push_back(o);
    o = align_up(o + plan(t[j].grid, s, t[j].nsrc).total);
  }
  *total = o;
  return EMM_OK;
}

struct PersistRun {
  std::vector<Prepared> P;
  std::unique_ptr<PSet> S;
  unsigned ctas = 0;
  size_t smem = 0;
  int rd = 0, shape = 0;
};

template <int R, int SH>
cudaError_t persist_shape(PersistRun *run, const emm_persist_opts &o) {
  const size_t sb = smem_bytes<R, SH>();
  cudaError_t e =
      cudaFuncSetAttribute(k_persist<R, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sb));
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<R, SH>, NT, sb);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (o.ctas_per_sm > 0) per_sm = std::min(per_sm, o.ctas_per_sm);
  long long g = static_cast<long long>(per_sm) * run->P[0].sms;
  if (o.max_ctas > 0) g = std::min<long long>(g, o.max_ctas);
  g = std::max<long long>(1, std::min<long long>(g, run->S->cta0[run->S->njobs]));
  run->ctas = static_cast<unsigned>(g);
  run->smem = sb;
  for (int j = 0; j < run->S->njobs; ++j) {
    PJob &J = run->S->job[j];
    if (!make_tiles<R, SH>(&J.tmE, J.p.H, J.p) || !make_tiles<R, SH>(&J.tmH, J.p.E, J.p))
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// Validate, prepare every task (enqueued on cs) and fill the launch
// parameters; steps_cap < 0: each task's own step count.
int persist_prepare(int nt, const emm_task *t, const emm_persist_opts *opts, void *ws, size_t ws_bytes,
                    cudaStream_t cs, bool upload, int steps_cap, PersistRun *run) {
  std::vector<size_t> off;
  size_t total = 0;
  int st = persist_layout(nt, t, &off, &total);
  if (st != EMM_OK) return st;
  emm_persist_opts o{0, 0, 0.0, -1, 0};
  if (opts) o = *opts;
  if (o.ctas_per_sm < 0 || o.max_ctas < 0 || o.tile_shape < 0 || o.tile_shape >= kShapes) return EMM_EINVAL;
  if (!ws || ws_bytes < total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return EMM_EWORKSPACE;
  for (int j = 0; j < nt; ++j)
    if (!t[j].sigma || (t[j].survey->nrec > 0 && !t[j].rec_out)) return EMM_EINVAL;
  unsigned char *base = static_cast<unsigned char *>(ws);
  if (cudaMemsetAsync(ws, 0, kAlign, cs) != cudaSuccess) return EMM_ECUDA;
  run->P.assign(nt, Prepared{});
  run->S.reset(new (std::nothrow) PSet{});
  if (!run->S) return EMM_ENOMEM;
  PSet &S = *run->S;
  int cta = 0, nmax = 0;
  for (int j = 0; j < nt; ++j) {
    const size_t end = j + 1 < nt ? off[j + 1] : total;
    st = prepare_forward(t[j].grid, t[j].survey, t[j].sigma, base + off[j], end - off[j], t[j].rec_out, nullptr, cs,
                         &run->P[j], t[j].nsrc, t[j].src_pos, false, upload, o.tile_shape);
    if (st != EMM_OK) return st;
    const Prepared &P = run->P[j];
    PJob &J = S.job[j];
    J.p = P.p;
    J.bx = static_cast<int>(P.blocks.x);
    J.by = static_cast<int>(P.blocks.y);
    J.nt = steps_cap >= 0 ? std::min(steps_cap, t[j].survey->nt) : t[j].survey->nt;
    S.cta0[j] = cta;
    cta += static_cast<int>(P.blocks.x * P.blocks.y * P.blocks.z);
    nmax = std::max(nmax, J.nt);
  }
  S.cta0[nt] = cta;
  S.njobs = nt;
  S.nt_max = nmax;
  S.status = reinterpret_cast<int *>(base + kPHdrStatus);
  S.abort = reinterpret_cast<int *>(base + kPHdrAbort);
  S.bar = reinterpret_cast<unsigned *>(base + kPHdrBar);
  S.claim = reinterpret_cast<unsigned long long *>(base + kPHdrClaim);
  for (int j = 0; j < nt; ++j) S.job[j].p.abort = S.abort;  // a tile wait that runs out stops the run
  S.wait_ns = static_cast<unsigned long long>((o.wait_s > 0 ? o.wait_s : 1.0) * 1e9);
  S.skip = o.skip_arrival;
  run->rd = run->P[0].rd;
  run->shape = o.tile_shape;
  cudaError_t e;
  const int key = 2 * run->rd + run->shape;
  switch (key) {
    case 2: e = persist_shape<1, 0>(run, o); break;
    case 3: e = persist_shape<1, 1>(run, o); break;
    case 4: e = persist_shape<2, 0>(run, o); break;
    case 5: e = persist_shape<2, 1>(run, o); break;
    case 6: e = persist_shape<3, 0>(run, o); break;
    case 7: e = persist_shape<3, 1>(run, o); break;
    case 8: e = persist_shape<4, 0>(run, o); break;
    default: e = persist_shape<4, 1>(run, o); break;
  }
  return e == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

// One cooperative launch of the prepared work list: every CTA resident.
cudaError_t persist_launch(const PersistRun &run, cudaStream_t cs) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(run.ctas);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = run.smem;
  cfg.stream = cs;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (2 * run.rd + run.shape) {
    case 2: return cudaLaunchKernelEx(&cfg, k_persist<1, 0>, *run.S);
    case 3: return cudaLaunchKernelEx(&cfg, k_persist<1, 1>, *run.S);
    case 4: return cudaLaunchKernelEx(&cfg, k_persist<2, 0>, *run.S);
    case 5: return cudaLaunchKernelEx(&cfg, k_persist<2, 1>, *run.S);
    case 6: return cudaLaunchKernelEx(&cfg, k_persist<3, 0>, *run.S);
    case 7: return cudaLaunchKernelEx(&cfg, k_persist<3, 1>, *run.S);
    case 8: return cudaLaunchKernelEx(&cfg, k_persist<4, 0>, *run.S);
    default: return cudaLaunchKernelEx(&cfg, k_persist<4, 1>, *run.S);
  }
}

int persist_finalize(const PersistRun &run, int nt, const emm_task *t, cudaStream_t cs) {
  for (int j = 0; j < nt; ++j) {
    const int st = finalize_forward(run.P[j], t[j].survey, t[j].rec_out, nullptr, cs);
    if (st != EMM_OK) return st;
  }
  return EMM_OK;
}

// ---- wavefront solve (k_wave) ----
// Workspace: the forward workspace, then the layer-item order (one unsigned
// per layer item) and the counters (cntE[L], cntH[L], cntR[2], the claim
// counter), 256-byte aligned.
struct WaveGeom {
  int L = 0, T = 0, RT = 0, a = 0, la = 0, lb = -1, K = 0, h = 0, rec_layers = 0;
  size_t nlayer = 0;
};

// gap: extra positions between an item and the items it waits for, so that
// with G CTAs in flight (about G / T layer items) a claimed item rarely finds
// its inputs still being computed; it changes the order, not the sizes.
int wave_geom(const emm_grid *g, const emm_survey *s, int depth, WaveGeom *w, int gap = 0) {
  const int st = check_survey(g, s);
  if (st != EMM_OK) return st;
  if (depth < 1 || depth > 64 || s->volume || s->airwave || s->src_kind != 0 || s->src_length > 0 ||
      s->nt >= (1 << 18))
    return EMM_EINVAL;
  const FieldGeom fg = field_geom(g, 0);
  const int rd = g->rd, zc = shape_zc(0);
  w->L = fg.tiles[2];
  w->T = fg.tiles[0] * fg.tiles[1];
  if (w->L > 4095) return EMM_EINVAL;
  w->a = (rd + zc - 1) / zc;
  // receiver CTAs (one warp per receiver component, 4 warps a CTA), in
  // layers of T CTA items, and the z-layers their stencils touch
  const int rec_blocks = (s->nrec * 3 + NT / 32 - 1) / (NT / 32);
  w->rec_layers = s->nrec > 0 ? (rec_blocks + w->T - 1) / w->T : 0;
  w->RT = w->rec_layers * w->T;
  if (s->nrec > 0) {
    int kmin = 1 << 30, kmax = -1;
    std::vector<double> wt(2 * static_cast<size_t>(rd));
    for (int r = 0; r < s->nrec; ++r)
      for (int c = 0; c < 6; ++c) {
        int k0 = 0;
        const int e = locate_axis(g, 2, kHalf[c][2], s->rec[3 * r + 2], &k0, wt.data());
        if (e != EMM_OK) return e;
        kmin = std::min(kmin, k0);
        kmax = std::max(kmax, k0 + 2 * rd - 1);
      }
    w->la = (kmin - fg.org[2]) / zc;
    w->lb = (kmax - fg.org[2]) / zc;
  }
  w->h = w->a + 1 + gap;
  w->K = std::max(w->a + w->h + 1 + gap, w->lb - w->la + 2 + gap);
  // layer items: per step L E items, L H items and 2 rec_layers receiver items
  w->nlayer = static_cast<size_t>(s->nt) * (2 * static_cast<size_t>(w->L) + 2 * w->rec_layers);
  (void)depth;
  return EMM_OK;
}

size_t wave_extra_bytes(const WaveGeom &w) {
  // counters: cntE[L], cntH[L], cntR[2], the 8-byte claim counter, the abort word
  return align_up(w.nlayer * sizeof(unsigned)) + align_up((2 * static_cast<size_t>(w.L) + 2) * sizeof(unsigned) + 16);
}

// The global order of the layer items: sweeps of `depth` steps; in a sweep
// starting at step s0, position q holds (in this order) the H receivers of
// step s0 + d if q == la + K d + h - 1, E(s0 + d, q - K d), H(s0 + d, q - K d
// - h) and the E receivers of step s0 + d if q == lb + K d + 1, for every d.
void wave_order(const WaveGeom &w, int nt, int depth, std::vector<unsigned> *out) {
  out->clear();
  out->reserve(w.nlayer);
  auto put = [&](int kind, int l, int s) {
    out->push_back(static_cast<unsigned>(kind) | (static_cast<unsigned>(l) << 2) | (static_cast<unsigned>(s) << 14));
  };
  for (int s0 = 0; s0 < nt; s0 += depth) {
    const int D = std::min(depth, nt - s0);
    const int qmax = w.L - 1 + w.K * (D - 1) + w.h;
    for (int q = 0; q <= qmax; ++q)
      for (int d = 0; d < D; ++d) {
        const int s = s0 + d;
        if (w.rec_layers && q == w.la + w.K * d + w.h - 1)
          for (int r = 0; r < w.rec_layers; ++r) put(2, r, s);
        const int le = q - w.K * d, lh = q - w.K * d - w.h;
        if (le >= 0 && le < w.L) put(0, le, s);
        if (lh >= 0 && lh < w.L) put(1, lh, s);
        if (w.rec_layers && q == w.lb + w.K * d + 1)
          for (int r = 0; r < w.rec_layers; ++r) put(3, r, s);
      }
  }
}

struct WaveRun {
  Prepared P;
  std::unique_ptr<WaveSet> W;
  unsigned ctas = 0;
  size_t smem = 0;
};

template <int R>
cudaError_t wave_shape(WaveRun *run) {
  const size_t sb = smem_bytes<R>();
  cudaError_t e = cudaFuncSetAttribute(k_wave<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sb));
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wave<R>, NT, sb);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  run->ctas = static_cast<unsigned>(per_sm * run->P.sms);
  run->smem = sb;
  WaveSet &W = *run->W;
  if (!make_tiles<R>(&W.tmE, W.p.H, W.p) || !make_tiles<R>(&W.tmH, W.p.E, W.p)) return cudaErrorInvalidValue;
  return cudaSuccess;
}

int wave_prepare(const emm_grid *g, const emm_survey *s, const float *sigma, int depth, void *ws, size_t ws_bytes,
                 double *rec_out, cudaStream_t cs, WaveRun *run) {
  WaveGeom w;
  int st = wave_geom(g, s, depth, &w);
  if (st != EMM_OK) return st;
  {
    // the CTAs in flight cover about G / T layer items, 2 per step of the
    // sweep and position: keep the waits at least that many positions back
    int sms = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int G = sms * min_ctas(g->rd), D = std::max(1, std::min(depth, s->nt));
    const int gap = (G + 2 * D * w.T - 1) / (2 * D * w.T);
    st = wave_geom(g, s, depth, &w, gap);
    if (st != EMM_OK) return st;
  }
  const size_t fwd = align_up(plan(g, s).total);
  if (!ws || ws_bytes < fwd + wave_extra_bytes(w) || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0)
    return EMM_EWORKSPACE;
  std::vector<unsigned> order;
  try {
    wave_order(w, s->nt, depth, &order);
  } catch (const std::bad_alloc &) {
    return EMM_ENOMEM;
  }
  if (order.size() != w.nlayer) return EMM_EINVAL;
  st = prepare_forward(g, s, sigma, ws, fwd, rec_out, nullptr, cs, &run->P, 1, nullptr, false, true, 0);
  if (st != EMM_OK) return st;
  if (run->P.p.rec_layers != w.rec_layers || run->P.p.tiles_z != w.L) return EMM_EINVAL;
  unsigned char *base = static_cast<unsigned char *>(ws) + fwd;
  unsigned *ord = reinterpret_cast<unsigned *>(base);
  unsigned *cnt = reinterpret_cast<unsigned *>(base + align_up(w.nlayer * sizeof(unsigned)));
  const size_t cnt_bytes = (2 * static_cast<size_t>(w.L) + 2) * sizeof(unsigned) + 8 + 8;  // + claim + abort
  cudaError_t e = cudaMemcpyAsync(ord, order.data(), order.size() * sizeof(unsigned), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, align_up(cnt_bytes), cs);
  if (e != cudaSuccess) return EMM_ECUDA;
  run->W.reset(new (std::nothrow) WaveSet{});
  if (!run->W) return EMM_ENOMEM;
  WaveSet &W = *run->W;
  W.p = run->P.p;
  W.order = ord;
  W.T = w.T;
  W.RT = w.RT;
  W.nitems = static_cast<long long>(w.nlayer) * w.T;
  W.a = w.a;
  W.la = w.la;
  W.lb = w.lb;
  W.L = w.L;
  W.cntE = cnt;
  W.cntH = cnt + w.L;
  W.cntR = cnt + 2 * w.L;
  W.claim = reinterpret_cast<unsigned long long *>(cnt + 2 * w.L + 2);
  W.status = W.p.status;
  W.abort = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(W.claim) + 8);  // after the claim counter
  W.p.abort = W.abort;
  W.wait_ns = 1000000000ull;
  switch (run->P.rd) {
    case 1: e = wave_shape<1>(run); break;
    case 2: e = wave_shape<2>(run); break;
    case 3: e = wave_shape<3>(run); break;
    default: e = wave_shape<4>(run); break;
  }
  return e == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

cudaError_t wave_launch(const WaveRun &run, cudaStream_t cs) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(run.ctas);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = run.smem;
  cfg.stream = cs;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (run.P.rd) {
    case 1: return cudaLaunchKernelEx(&cfg, k_wave<1>, *run.W);
    case 2: return cudaLaunchKernelEx(&cfg, k_wave<2>, *run.W);
    case 3: return cudaLaunchKernelEx(&cfg, k_wave<3>, *run.W);
    default: return cudaLaunchKernelEx(&cfg, k_wave<4>, *run.W);
  }
}

int finalize_forward(const Prepared &P, const emm_survey *s, double *rec_out, double *vol_out, cudaStream_t cs) {
  const int nf = s->nfreq;
  const double *dnorm = reinterpret_cast<const double *>(reinterpret_cast<const unsigned char *>(P.p.status) -
                                                         P.L.status + P.L.norm);
  if (s->nrec > 0) {
    const int nr = P.p.nsrc * s->nrec, tot = nr * 6 * nf;
    k_finalize_rec<<<(tot + 255) / 256, 256, 0, cs>>>(rec_out, dnorm, nr, nf);
  }
  if (s->volume) {
    const size_t nint = static_cast<size_t>(P.p.n[0]) * P.p.n[1] * P.p.n[2];
    k_finalize_vol<<<8 * P.sms, 256, 0, cs>>>(P.p.vacc, vol_out, dnorm, nint, nf);
  }
  return cudaGetLastError() == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

int forward_impl(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                 double *rec_out, double *vol_out, emm_stream stream, StepEvents *te) {
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  Prepared P;
  int st = prepare_forward(g, s, sigma, ws, ws_bytes, rec_out, vol_out, cs, &P);
  if (st != EMM_OK) return st;
  if (run_steps(P, P.p, P.blocks, 0, s->nt, cs, te) != cudaSuccess) return EMM_ECUDA;
  return finalize_forward(P, s, rec_out, vol_out, cs);
}

// cuCtxGetCurrent, fetched once from the driver through the runtime.
static PFN_cuCtxGetCurrent_v4000 context_query() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
  });
  return fn;
}

// Device address of emm_static_scratch in the current context, looked up
// with that context current and cached per context.  A device reset (or any
// context teardown) loads the module again into a new context, where the
// array may sit at another address: that context gets a lookup of its own.
static int static_scratch(void **ptr) {
  constexpr int kSlots = 64;
  static std::mutex mu;
  static CUcontext ctx[kSlots] = {};
  static void *addr[kSlots] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return EMM_ECUDA;
  PFN_cuCtxGetCurrent_v4000 get = context_query();
  CUcontext cur = nullptr;
  if (!get || get(&cur) != CUDA_SUCCESS) return EMM_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  const int slot = dev % kSlots;
  if (cur && ctx[slot] == cur && addr[slot]) {
    *ptr = addr[slot];
    return EMM_OK;
  }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, emm_static_scratch) != cudaSuccess || !p) return EMM_ECUDA;
  // a thread with no current context gets the device's primary context from
  // the lookup above
  if (!cur && (get(&cur) != CUDA_SUCCESS || !cur)) return EMM_ECUDA;
  ctx[slot] = cur;
  addr[slot] = p;
  *ptr = p;
  return EMM_OK;
}

}  // namespace emm

using namespace emm;

extern "C" {

int emm_workspace_size(const emm_grid *g, const emm_survey *s, size_t *bytes) {
  const int st = check_survey(g, s);
  if (st != EMM_OK) return st;
  if (!bytes) return EMM_EINVAL;
  *bytes = plan(g, s).total;
  return EMM_OK;
}

int emm_forward(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                double *rec_out, double *vol_out, emm_stream stream) {
  return forward_impl(g, s, sigma, ws, ws_bytes, rec_out, vol_out, stream, nullptr);
}

int emm_forward_timed(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                      double *rec_out, double *vol_out, emm_stream stream, emm_timing *timing) {
  if (!timing || timing->every < 1) return EMM_EINVAL;
  int st = check_survey(g, s);
  if (st != EMM_OK) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int nsamp = s->nt > 0 ? (s->nt + timing->every - 1) / timing->every : 0;
  std::vector<cudaEvent_t> all(4 * static_cast<size_t>(nsamp) + 4, nullptr);
  for (auto &e : all)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto &d : all)
        if (d) cudaEventDestroy(d);
      return EMM_ECUDA;
    }
  StepEvents te;
  te.every = timing->every;
  te.ev.assign(all.begin(), all.begin() + 4 * static_cast<size_t>(nsamp));
  cudaEvent_t t0 = all[all.size() - 2], t1 = all[all.size() - 1];
  te.loop[0] = all[all.size() - 4];
  te.loop[1] = all[all.size() - 3];
  cudaEventRecord(t0, cs);
  st = forward_impl(g, s, sigma, ws, ws_bytes, rec_out, vol_out, stream, &te);
  cudaEventRecord(t1, cs);
  if (cudaStreamSynchronize(cs) != cudaSuccess && st == EMM_OK) st = EMM_ECUDA;
  double se = 0, sv = 0, sh = 0;
  long vsteps = 0;
  float ms = 0.f;
  const int taken = std::min(te.used, nsamp);
  for (int q = 0; q < taken && st == EMM_OK; ++q) {
    cudaEventElapsedTime(&ms, te.ev[4 * q], te.ev[4 * q + 1]);
    se += ms;
    cudaEventElapsedTime(&ms, te.ev[4 * q + 1], te.ev[4 * q + 2]);
    sv += ms;
    vsteps += q < static_cast<int>(te.vsteps.size()) ? te.vsteps[q] : 0;
    cudaEventElapsedTime(&ms, te.ev[4 * q + 2], te.ev[4 * q + 3]);
    sh += ms;
  }
  // per step: the E and H launches of the timed steps; the volume DTFT
  // launches of those steps over the steps they covered
  timing->samples = taken;
  timing->e_ms = taken ? se / taken : 0.0;
  timing->v_ms = (vsteps > 0 && s->volume) ? sv / static_cast<double>(vsteps) : 0.0;
  timing->h_ms = taken ? sh / taken : 0.0;
  ms = 0.f;
  if (st == EMM_OK) cudaEventElapsedTime(&ms, t0, t1);
  timing->total_ms = ms;
  ms = 0.f;
  if (st == EMM_OK && s->nt > 0) cudaEventElapsedTime(&ms, te.loop[0], te.loop[1]);
  timing->loop_ms = ms;
  for (auto &e : all) cudaEventDestroy(e);
  return st;
}

int emm_forward_converge(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                         double *rec_out, double *vol_out, emm_stream stream, int *nt_run) {
  using namespace emm;
  if (!nt_run) return EMM_EINVAL;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  Prepared P;
  int st = prepare_forward(g, s, sigma, ws, ws_bytes, rec_out, vol_out, cs, &P, 1, nullptr, true);
  if (st != EMM_OK) return st;
  // The verdicts come back through mapped host memory (Sec. 4.1): [0] the
  // last step checked, [1] the steps to keep once converged.
  int *hw = nullptr, *dw = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void **>(&hw), 2 * sizeof(int), cudaHostAllocMapped) != cudaSuccess)
    return EMM_ECUDA;
  volatile int *vhw = hw;
  vhw[0] = -1;
  vhw[1] = 0;
  if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&dw), hw, 0) != cudaSuccess) {
    cudaFreeHost(hw);
    return EMM_ECUDA;
  }
  int *halt = const_cast<int *>(P.p.halt);
  // Chunks: step 0, then the reference corner values; then up to and
  // including each step it = 100, 200, ... and its check; then the rest.
  const int nt = s->nt;
  struct Chunk {
    int lo, hi, check;  // steps lo .. hi-1, then the check after step `check` (-1: none)
  };
  std::vector<Chunk> chunks;
  if (nt > 0) chunks.push_back({0, 1, 0});
  for (int it = 100; it < nt; it += 100) chunks.push_back({chunks.back().hi, it + 1, it});
  if (!chunks.empty() && chunks.back().hi < nt) chunks.push_back({chunks.back().hi, nt, -1});
  auto enqueue = [&](const Chunk &c) {
    cudaError_t e = run_steps(P, P.p, P.blocks, c.lo, c.hi, cs, nullptr);
    if (e == cudaSuccess && c.check >= 0) {
      k_corner_check<<<1, 32, 0, cs>>>(P.p.corner, halt, dw, c.check, c.check == 0 ? 1 : 0);
      e = cudaGetLastError();
    }
    return e;
  };
  // One chunk of look-ahead: chunk q+1 is enqueued before the host waits
  // (bounded) for the verdict of chunk q; launches after a stop return at once.
  // bound of one wait for a verdict; EMM_POLL_TIMEOUT_S (seconds) lowers it
  // for tests of the timeout path
  double poll_s = 600.0;
  if (const char *env = std::getenv("EMM_POLL_TIMEOUT_S")) {
    const double v = std::atof(env);
    if (v > 0) poll_s = v;
  }
  size_t next = 0;
  bool stopped = false;
  for (size_t q = 0; q < chunks.size() && st == EMM_OK && !stopped; ++q) {
    while (next < chunks.size() && next <= q + 1 && st == EMM_OK)
      if (enqueue(chunks[next++]) != cudaSuccess) st = EMM_ECUDA;
    if (st != EMM_OK || chunks[q].check < 0) continue;
    const auto t0 = std::chrono::steady_clock::now();
    while (vhw[0] < chunks[q].check) {
      if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > poll_s) {
        st = EMM_ETIMEOUT;
        break;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    if (vhw[1] > 0) stopped = true;
  }
  if (cudaStreamSynchronize(cs) != cudaSuccess && st == EMM_OK) st = EMM_ECUDA;
  const int kept = vhw[1] > 0 ? vhw[1] : nt;
  cudaFreeHost(hw);
  if (st != EMM_OK) return st;
  // normalisation over the steps taken
  std::vector<double> norm(4 * static_cast<size_t>(s->nfreq));
  normalisation(s, P.dt, kept, norm.data());
  unsigned char *base = static_cast<unsigned char *>(ws);
  if (cudaMemcpy(base + P.L.norm, norm.data(), norm.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return EMM_ECUDA;
  st = finalize_forward(P, s, rec_out, vol_out, cs);
  if (st == EMM_OK && cudaStreamSynchronize(cs) != cudaSuccess) st = EMM_ECUDA;
  *nt_run = kept;
  return st;
}

int emm_jobs_workspace_size(int njobs, const emm_job *jobs, size_t *bytes, size_t *offsets) {
  if (!bytes) return EMM_EINVAL;
  std::vector<size_t> off;
  const int st = emm::jobs_layout(njobs, jobs, &off, bytes);
  if (st != EMM_OK) return st;
  if (offsets)
    for (int j = 0; j < njobs; ++j) offsets[j] = off[j];
  return EMM_OK;
}

int emm_forward_jobs(int njobs, const emm_job *jobs, int strategy, void *ws, size_t ws_bytes, emm_stream stream) {
  return emm::forward_jobs_impl(njobs, jobs, strategy, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

int emm_jobs_tune(int njobs, const emm_job *jobs, void *ws, size_t ws_bytes, int steps, emm_stream stream,
                  double *ms, int *best) {
  return emm::jobs_tune(njobs, jobs, ws, ws_bytes, steps, reinterpret_cast<cudaStream_t>(stream), ms, best);
}

int emm_wave_workspace_size(const emm_grid *g, const emm_survey *s, int depth, size_t *bytes) {
  if (!bytes) return EMM_EINVAL;
  emm::WaveGeom w;
  const int st = emm::wave_geom(g, s, depth, &w);
  if (st != EMM_OK) return st;
  *bytes = emm::align_up(emm::plan(g, s).total) + emm::wave_extra_bytes(w);
  return EMM_OK;
}

int emm_forward_wave(const emm_grid *g, const emm_survey *s, const float *sigma, int depth, void *ws,
                     size_t ws_bytes, double *rec_out, emm_stream stream) {
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::WaveRun run;
  int st = emm::wave_prepare(g, s, sigma, depth, ws, ws_bytes, rec_out, cs, &run);
  if (st != EMM_OK) return st;
  if (emm::wave_launch(run, cs) != cudaSuccess) return EMM_ECUDA;
  return emm::finalize_forward(run.P, s, rec_out, nullptr, cs);
}

int emm_persist_workspace_size(int ntasks, const emm_task *tasks, size_t *bytes, size_t *offsets) {
  if (!bytes) return EMM_EINVAL;
  std::vector<size_t> off;
  const int st = emm::persist_layout(ntasks, tasks, &off, bytes);
  if (st != EMM_OK) return st;
  if (offsets)
    for (int j = 0; j < ntasks; ++j) offsets[j] = off[j];
  return EMM_OK;
}

int emm_forward_persistent(int ntasks, const emm_task *tasks, const emm_persist_opts *opts, void *ws,
                           size_t ws_bytes, emm_stream stream) {
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::PersistRun run;
  int st = emm::persist_prepare(ntasks, tasks, opts, ws, ws_bytes, cs, true, -1, &run);
  if (st != EMM_OK) return st;
  if (emm::persist_launch(run, cs) != cudaSuccess) return EMM_ECUDA;
  return emm::persist_finalize(run, ntasks, tasks, cs);
}

int emm_persist_tune(int ntasks, const emm_task *tasks, void *ws, size_t ws_bytes, int steps, emm_stream stream,
                     int *ncand, emm_persist_opts *cands, double *ms, emm_persist_opts *best) {
  if (steps < 1 || !ncand || *ncand < 1 || !cands || !ms || !best) return EMM_EINVAL;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::PersistRun run;
  // the candidates: each tile shape with 1 .. its occupancy limit of
  // resident CTAs per SM, in that order, at most *ncand of them
  std::vector<emm_persist_opts> cand;
  int st = EMM_OK;
  for (int sh = 0; sh < emm::kShapes && st == EMM_OK; ++sh) {
    const emm_persist_opts probe{0, 0, 0.0, -1, sh};
    st = emm::persist_prepare(ntasks, tasks, &probe, ws, ws_bytes, cs, sh == 0, steps, &run);
    const int top = st == EMM_OK ? static_cast<int>((run.ctas + run.P[0].sms - 1) / run.P[0].sms) : 0;
    for (int k = 1; k <= top; ++k) cand.push_back(emm_persist_opts{k, 0, 0.0, -1, sh});
  }
  if (st != EMM_OK) return st;
  const int nc = std::min(static_cast<int>(cand.size()), *ncand);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return EMM_ECUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return EMM_ECUDA;
  }
  int bi = -1;
  for (int k = 0; k < nc && st == EMM_OK; ++k) {
    for (int rep = 0; rep < 2 && st == EMM_OK; ++rep) {  // a warm-up run, then the timed one
      st = emm::persist_prepare(ntasks, tasks, &cand[k], ws, ws_bytes, cs, false, steps, &run);
      if (st == EMM_OK && rep == 1 && cudaEventRecord(a, cs) != cudaSuccess) st = EMM_ECUDA;
      if (st == EMM_OK && emm::persist_launch(run, cs) != cudaSuccess) st = EMM_ECUDA;
      if (st == EMM_OK && rep == 1 && cudaEventRecord(b, cs) != cudaSuccess) st = EMM_ECUDA;
    }
    float t = 0.f;
    if (st == EMM_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess))
      st = EMM_ECUDA;
    cands[k] = cand[k];
    ms[k] = t;
    if (st == EMM_OK && (bi < 0 || t < ms[bi])) bi = k;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != EMM_OK) return st;
  *ncand = nc;
  *best = cand[bi];
  return EMM_OK;
}

}  // extern "C"

struct emm_persist_plan {
  std::vector<emm_task> tasks;
  std::vector<emm_survey> surveys;
  std::vector<std::vector<double>> recs, freqs, pos;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

int emm_persist_plan_create(int ntasks, const emm_task *tasks, const emm_persist_opts *opts, void *ws,
                            size_t ws_bytes, emm_stream stream, emm_persist_plan **out) {
  if (!out) return EMM_EINVAL;
  *out = nullptr;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  // a first set-up on the caller's stream uploads the tables the graph's
  // runs then find in the workspace
  emm::PersistRun run;
  int st = emm::persist_prepare(ntasks, tasks, opts, ws, ws_bytes, cs, true, -1, &run);
  if (st != EMM_OK) return st;
  std::unique_ptr<emm_persist_plan> pl(new (std::nothrow) emm_persist_plan);
  if (!pl) return EMM_ENOMEM;
  // the plan's own copies of what the tasks point to on the host
  pl->tasks.assign(tasks, tasks + ntasks);
  pl->surveys.resize(ntasks);
  pl->recs.resize(ntasks);
  pl->freqs.resize(ntasks);
  pl->pos.resize(ntasks);
  for (int j = 0; j < ntasks; ++j) {
    const emm_survey *s = tasks[j].survey;
    pl->surveys[j] = *s;
    pl->recs[j].assign(s->rec, s->rec + (s->nrec > 0 ? 3 * static_cast<size_t>(s->nrec) : 0));
    pl->freqs[j].assign(s->freqs, s->freqs + s->nfreq);
    pl->surveys[j].rec = pl->recs[j].empty() ? nullptr : pl->recs[j].data();
    pl->surveys[j].freqs = pl->freqs[j].data();
    pl->tasks[j].survey = &pl->surveys[j];
    if (tasks[j].src_pos) {
      pl->pos[j].assign(tasks[j].src_pos, tasks[j].src_pos + 3 * static_cast<size_t>(tasks[j].nsrc));
      pl->tasks[j].src_pos = pl->pos[j].data();
    }
  }
  // capture on a stream of the plan's own: the set-up without the table
  // upload, the cooperative launch and the normalisation
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    emm::PersistRun r2;
    st = emm::persist_prepare(ntasks, pl->tasks.data(), opts, ws, ws_bytes, cap, false, -1, &r2);
    if (st == EMM_OK && emm::persist_launch(r2, cap) != cudaSuccess) st = EMM_ECUDA;
    if (st == EMM_OK) st = emm::persist_finalize(r2, ntasks, pl->tasks.data(), cap);
    e = cudaStreamEndCapture(cap, &graph);
  }
  if (e == cudaSuccess && st == EMM_OK) e = cudaGraphInstantiate(&pl->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  if (st != EMM_OK) return st;
  if (e != cudaSuccess) return EMM_ECUDA;
  *out = pl.release();
  return EMM_OK;
}

int emm_persist_plan_run(emm_persist_plan *pl, emm_stream stream) {
  if (!pl || !pl->exec) return EMM_EINVAL;
  return cudaGraphLaunch(pl->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

void emm_persist_plan_destroy(emm_persist_plan *pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  delete pl;
}

int emm_batch_workspace_size(const emm_grid *g, const emm_survey *s, int nsrc, size_t *bytes) {
  const int st = emm::check_survey(g, s);
  if (st != EMM_OK) return st;
  if (!bytes || nsrc < 1 || s->volume) return EMM_EINVAL;
  *bytes = emm::plan(g, s, nsrc).total;
  return EMM_OK;
}

int emm_forward_batch(const emm_grid *g, const emm_survey *s, int nsrc, const double *src_pos, const float *sigma,
                      void *ws, size_t ws_bytes, double *rec_out, emm_stream stream) {
  if (nsrc < 1 || !src_pos) return EMM_EINVAL;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::Prepared P;
  int st = emm::prepare_forward(g, s, sigma, ws, ws_bytes, rec_out, nullptr, cs, &P, nsrc, src_pos);
  if (st != EMM_OK) return st;
  if (emm::run_steps(P, P.p, P.blocks, 0, s->nt, cs, nullptr) != cudaSuccess) return EMM_ECUDA;
  return emm::finalize_forward(P, s, rec_out, nullptr, cs);
}

int emm_forward_static(const emm_grid *g, const emm_survey *s, const float *sigma, double *rec_out,
                       double *vol_out, emm_stream stream, int *status) {
  int st = emm::check_survey(g, s);
  if (st != EMM_OK) return st;
  if (emm::plan(g, s).total > EMM_STATIC_SCRATCH_BYTES) return EMM_EWORKSPACE;
  void *ws = nullptr;
  st = emm::static_scratch(&ws);
  if (st != EMM_OK) return st;
  st = emm::forward_impl(g, s, sigma, ws, EMM_STATIC_SCRATCH_BYTES, rec_out, vol_out, stream, nullptr);
  if (st == EMM_OK && status) st = emm_status(ws, status, stream);
  return st;
}

int emm_status(const void *ws, int *status, emm_stream stream) {
  if (!ws || !status) return EMM_EINVAL;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess) return EMM_ECUDA;
  if (cudaStreamSynchronize(cs) != cudaSuccess) return EMM_ECUDA;
  *status = v;
  return EMM_OK;
}

}  // extern "C"
