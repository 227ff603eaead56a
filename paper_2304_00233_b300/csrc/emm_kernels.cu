// emm_kernels.cu -- sm_103a kernels of the fictitious-wave FDTD time loop and
// the emm_forward / emm_forward_timed / emm_workspace_size / emm_status
// entry points.
//
// One leapfrog step (Algorithm 1 without the airwave step) is two launches:
//
//   k_update_E<R>  curl H with D- rows and CPML memory (Eq. 14, 22-24), the
//                  electric source at t_{n+1/2}, E += dt/eps (curl H - J)
//                  (Eq. 8); extra CTAs accumulate the receiver DTFT of
//                  H^{n+1/2} (Eq. 25), which this launch only reads; interior
//                  threads accumulate the volume DTFT of H^{n+1/2}.
//   k_update_H<R>  curl E with D+ rows and CPML memory (Eq. 13, 22-24),
//                  H -= dt/mu0 curl E; extra CTAs accumulate the receiver
//                  DTFT of E^{n+1}; interior threads the volume DTFT of E^{n+1}.
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
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <vector>

#include "emm_internal.h"

// Scratch of emm_forward_static: one array per device for the process
// lifetime.  In host code this name only stands for the symbol; its device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char emm_static_scratch[EMM_STATIC_SCRATCH_BYTES];

namespace emm {
namespace {

constexpr int TX = 32;  // tile width (x, one warp)
constexpr int TY = 8;   // tile height (y)
constexpr int NT = TX * TY;
constexpr int ZC = 4;   // planes per CTA
constexpr int XH = 4;   // x halo of the TMA boxes (>= R; keeps box x starts 16-byte aligned)
constexpr int WX = TX + 2 * XH;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of the mbarrier wait

// Resident CTAs per SM the register budget is sized for.
__host__ __device__ constexpr int min_ctas(int R) { return R <= 2 ? 3 : 2; }

// Shared-memory tiles of one CTA, for either half-step.  "zf" is the source
// field with z and y halos (Hx / Ex), "xf" the one with z and x halos
// (Hy / Ey), "xy" the one with x and y halos (Hz / Ez).
template <int R>
struct Tiles {
  static constexpr int ZQ = ZC + 2 * R - 1;  // planes of the z-halo boxes
  static constexpr int YH = TY + 2 * R;      // rows of the y-halo boxes
  static constexpr int ZF = ZQ * YH * TX;
  static constexpr int XF = ZQ * TY * WX;
  static constexpr int XY = ZC * YH * WX;
  static constexpr size_t BYTES = static_cast<size_t>(ZF + XF + XY) * 4;  // the three TMA boxes
  static constexpr int PSI = 6 * ZC * NT;  // CPML memory staged per thread: [6 slots][ZC][NT]
  static constexpr size_t ALL = BYTES + static_cast<size_t>(PSI) * 4;
};
template <int R>
constexpr size_t smem_bytes() { return Tiles<R>::ALL + 144; }  // + alignment pad + mbarrier

// Tensor maps of one launch: the three source fields with their boxes.
struct TmaSet {
  CUtensorMap m[3];
};

// ---- PTX helpers: mbarrier and TMA ---------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of `bar` for at most kWaitNs; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, uint64_t *bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// 4-byte asynchronous global -> shared copy (completes at cp_async_wait_all).
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ int slab_int(int i, int np, int nb) {
  return i < nb ? i : (i >= np - nb ? nb + np - 1 - i : -1);
}
__device__ __forceinline__ int slab_half(int i, int np, int nb) {
  return i < nb ? i : ((i >= np - 1 - nb && i <= np - 2) ? nb + np - 2 - i : -1);
}

// CPML memory array of a derivative along axis a: the slab (2nb entries)
// replaces that axis.  x: [np2][np1][2nb], y: [np2][2nb][np0], z: [2nb][np1][np0].
__device__ __forceinline__ size_t psi_at(int a, int s, int i, int j, int k, const int *np, int nb2) {
  if (a == 0) return (static_cast<size_t>(k) * np[1] + j) * nb2 + s;
  if (a == 1) return (static_cast<size_t>(k) * nb2 + s) * np[0] + i;
  return (static_cast<size_t>(s) * np[1] + j) * np[0] + i;
}

// CPML update of one derivative d (Eq. 22-23, kappa = 1): psi <- b psi + a d
// from the staged old value, stored back; returns d + psi.
__device__ __forceinline__ float cpml_step(float d, float old, float *__restrict__ psi, size_t idx, float a,
                                           float b) {
  const float v = fmaf(b, old, a * d);
  psi[idx] = v;
  return d + v;
}

// Stage this thread's CPML memory of planes k0 .. k0+ZC-1 into shared memory
// slots [slot][c][thread] with asynchronous copies.  Slots follow the psi
// arrays: 0 (y), 1 (z), 2 (z), 3 (x), 4 (x), 5 (y) derivative.  sx, sy are
// the x / y slab entries of the column (-1 outside), slab_k(k) the z entry.
template <class SlabK>
__device__ __forceinline__ void stage_psi(float *ps, float *const *psi, const DevParams &p, int i, int j, int k0,
                                          int sx, int sy, SlabK slab_k) {
  constexpr int S = ZC * NT;
  const int nb2 = 2 * p.nb;
#pragma unroll
  for (int c = 0; c < ZC; ++c) {
    const int k = k0 + c;
    if (k < 0) continue;
    if (k >= p.np[2]) break;
    const int sz = slab_k(k);
    float *d = ps + c * NT + threadIdx.x;
    if (sy >= 0) {
      const size_t id = psi_at(1, sy, i, j, k, p.np, nb2);
      cp_async4(d, psi[0] + id);
      cp_async4(d + 5 * S, psi[5] + id);
    }
    if (sz >= 0) {
      const size_t id = psi_at(2, sz, i, j, k, p.np, nb2);
      cp_async4(d + S, psi[1] + id);
      cp_async4(d + 2 * S, psi[2] + id);
    }
    if (sx >= 0) {
      const size_t id = psi_at(0, sx, i, j, k, p.np, nb2);
      cp_async4(d + 3 * S, psi[3] + id);
      cp_async4(d + 4 * S, psi[4] + id);
    }
  }
  cp_async_commit();
}

// Error-free accumulation (hi, lo) += v  (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v) {
  const float t = hi + v;
  const float bp = t - hi;
  const float err = (hi - (t - bp)) + (v - bp);
  hi = t;
  lo += err;
}

__device__ __forceinline__ void volume_accumulate(const DevParams &p, int comp, int lin, size_t nint,
                                                  const float *fac, float v) {
  for (int f = 0; f < p.nf; ++f) {
    float4 *a = p.vacc + (static_cast<size_t>(comp) * p.nf + f) * nint + lin;
    float4 acc = *a;
    two_sum_add(acc.x, acc.y, fac[2 * f] * v);
    two_sum_add(acc.z, acc.w, fac[2 * f + 1] * v);
    *a = acc;
  }
}

// One warp per (receiver, component): (2R)^3 weighted gather in FP64, warp
// shuffle reduction, then acc += factor * value for every frequency.
template <int R>
__device__ void receiver_dft(const DevParams &p, int comp0, float *const *F, const double *fac, int block) {
  constexpr int M = 2 * R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = block * (NT / 32) + warp;
  if (item >= p.nrec * 3) return;
  const int rec = item / 3, c = comp0 + item % 3;
  const int *st = p.rec_start + (rec * 6 + c) * 3;
  const double *w = p.rec_w + static_cast<size_t>(rec * 6 + c) * 3 * M;
  const float *f = F[c - comp0];
  double s = 0.0;
  for (int t = lane; t < M * M * M; t += 32) {
    const int q1 = t % M, q2 = (t / M) % M, q3 = t / (M * M);
    const size_t id = (static_cast<size_t>(st[2] + q3) * p.np[1] + (st[1] + q2)) * p.pitch + (st[0] + q1);
    s += w[q1] * w[M + q2] * w[2 * M + q3] * static_cast<double>(f[id]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double *acc = p.rec_acc + static_cast<size_t>(rec * 6 + c) * p.nf * 2;
    for (int q = 0; q < p.nf; ++q) {
      acc[2 * q] += fac[2 * q] * s;
      acc[2 * q + 1] += fac[2 * q + 1] * s;
    }
  }
}


// ---------------------------------------------------------------------------
// Common CTA prologue: origin of the tile, the TMA copies of the three source
// fields, and the bounded wait for them.
// ---------------------------------------------------------------------------
struct Origin {
  int i0, j0, k0;
};
__device__ __forceinline__ Origin origin_of(const DevParams &p, int b) {
  return Origin{p.org[0] + (b % p.tiles_x) * TX, p.org[1] + ((b / p.tiles_x) % p.tiles_y) * TY,
                p.org[2] + (b / (p.tiles_x * p.tiles_y)) * ZC};
}

// Shared-memory views of the three tiles (see Tiles).
template <int R>
struct View {
  using T = Tiles<R>;
  const float *s;
  __device__ float zf(int pz, int y, int x) const { return s[(pz * T::YH + y) * TX + x]; }
  __device__ float xf(int pz, int y, int x) const { return s[T::ZF + (pz * TY + y) * WX + x]; }
  __device__ float xy(int pz, int y, int x) const { return s[T::ZF + T::XF + (pz * T::YH + y) * WX + x]; }
};

// Thread 0: initialise the CTA's mbarrier and issue the three copies.  The
// z-halo boxes start `lead` planes from k0 (-R for D-, -R+1 for D+).
template <int R>
__device__ __forceinline__ void issue_tiles(const TmaSet &tm, float *s, uint64_t *bar, const Origin &o, int lead) {
  using T = Tiles<R>;
  mbar_init(bar, 1);
  fence_barrier_init();
  mbar_expect_tx(bar, static_cast<uint32_t>(T::BYTES));
  tma_load_3d(s, &tm.m[0], bar, o.i0, o.j0 - R, o.k0 + lead);
  tma_load_3d(s + T::ZF, &tm.m[1], bar, o.i0 - XH, o.j0, o.k0 + lead);
  tma_load_3d(s + T::ZF + T::XF, &tm.m[2], bar, o.i0 - XH, o.j0 - R, o.k0);
}

// All threads: wait for the copies.  False (after setting the status word
// and draining the copies, both bounded) if the wait ran out anywhere.
__device__ __forceinline__ bool tiles_ready(const DevParams &p, uint64_t *bar) {
  __syncthreads();  // the barrier is initialised
  const bool ok = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicExch(p.status, EMM_ETIMEOUT);
      mbar_wait_bounded(bar, 0);
    }
    __syncthreads();
    return false;
  }
  return true;
}

__device__ __forceinline__ float *smem_tiles(unsigned char *raw) {
  const uint32_t pad = (128u - (smem_u32(raw) & 127u)) & 127u;
  return reinterpret_cast<float *>(raw + pad);
}

// Does the CTA's box meet the bounding box of the source stencils?
__device__ __forceinline__ bool cta_has_source(const DevParams &p, const Origin &o) {
  return p.src_any && o.i0 + TX > p.src_lo[0] && o.i0 <= p.src_hi[0] && o.j0 + TY > p.src_lo[1] &&
         o.j0 <= p.src_hi[1] && o.k0 + ZC > p.src_lo[2] && o.k0 <= p.src_hi[2];
}

template <int R>
__device__ __forceinline__ void source_term(const DevParams &p, int c, int i, int j, int k, float amp,
                                            float &curl) {
  constexpr int M = 2 * R;
  if (!p.src_on[c]) return;
  const int a = i - p.src_start[c][0], bb = j - p.src_start[c][1], cc = k - p.src_start[c][2];
  if (a >= 0 && a < M && bb >= 0 && bb < M && cc >= 0 && cc < M) curl -= amp * p.jw[c][(cc * M + bb) * M + a];
}

// ---------------------------------------------------------------------------
// E half-step: E^{n+1} = E^n + dt/eps (curl H^{n+1/2} - J^{n+1/2})
// ---------------------------------------------------------------------------
// Is every cell of the CTA inside the CPML-free region where all D- rows
// exist (no slab, no boundary test needed)?
__device__ __forceinline__ bool interior_E(const DevParams &p, const Origin &o, int R) {
  const int m = max(p.nb, R);
  return o.i0 >= m && o.i0 + TX - 1 <= p.np[0] - 1 - m && o.j0 >= m && o.j0 + TY - 1 <= p.np[1] - 1 - m &&
         o.k0 >= m && o.k0 + ZC - 1 <= p.np[2] - 1 - m;
}

// The ZC planes of one column.  FAST: an interior CTA without the source,
// where every validity test is true and every slab test false.
template <int R, bool VOL, bool FAST>
__device__ __forceinline__ void e_planes(const DevParams &p, const View<R> &v, const Origin &o, int tx, int ty,
                                         const float (&e)[3][ZC], const float (&w)[3][ZC], const float *ps,
                                         int n, bool src) {
  constexpr int M = 2 * R;
  const int i = o.i0 + tx, j = o.j0 + ty;
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const size_t col = static_cast<size_t>(j) * p.pitch + i;
  const bool dm_i = FAST || (i >= R && i <= np0 - 1 - R), dm_j = FAST || (j >= R && j <= np1 - 1 - R);
  const int si = FAST ? -1 : slab_int(i, np0, nb), sj = FAST ? -1 : slab_int(j, np1, nb);
  float cx[M], cy[M];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    cx[q] = dm_i ? __ldg(p.cm[0] + i * M + q) : 0.f;
    cy[q] = dm_j ? __ldg(p.cm[1] + j * M + q) : 0.f;
  }
  const float amp = FAST ? 0.f : __ldg(p.amp + n);
  const int ii = i - p.nbe, jj = j - p.nbe;
  const bool int_ij = VOL && ii >= 0 && ii < p.n[0] && jj >= 0 && jj < p.n[1];
  const size_t nint = static_cast<size_t>(p.n[0]) * p.n[1] * p.n[2];
  const float *facH = p.fH32 + static_cast<size_t>(n) * p.nf * 2;

#pragma unroll
  for (int c = 0; c < ZC; ++c) {
    const int k = o.k0 + c;
    if (!FAST) {
      if (k < 0) continue;
      if (k >= np2) break;
    }
    const size_t id = static_cast<size_t>(k) * p.plane + col;
    const bool dm_k = FAST || (k >= R && k <= np2 - 1 - R);
    const int sk = FAST ? -1 : slab_int(k, np2, nb);
    float cz[M];
#pragma unroll
    for (int q = 0; q < M; ++q) cz[q] = dm_k ? __ldg(p.cm[2] + k * M + q) : 0.f;
    // Ex at (i+1/2, j, k): D-_y Hz - D-_z Hy
    if (FAST || (i <= np0 - 2 && dm_j && dm_k)) {
      float dy = 0.f, dz = 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        dy = fmaf(cy[q], v.xy(c, ty + q, tx + XH), dy);
        dz = fmaf(cz[q], v.xf(c + q, ty, tx + XH), dz);
      }
      if (!FAST) {
        if (sj >= 0)
          dy = cpml_step(dy, ps[(0 * ZC + c) * NT + threadIdx.x], p.psiE[0], psi_at(1, sj, i, j, k, p.np, 2 * nb),
                         p.pml[1][sj], p.pml[1][2 * nb + sj]);
        if (sk >= 0)
          dz = cpml_step(dz, ps[(1 * ZC + c) * NT + threadIdx.x], p.psiE[1], psi_at(2, sk, i, j, k, p.np, 2 * nb),
                         p.pml[2][sk], p.pml[2][2 * nb + sk]);
      }
      float curl = dy - dz;
      if (!FAST && src) source_term<R>(p, 0, i, j, k, amp, curl);
      p.E[0][id] = fmaf(w[0][c], curl, e[0][c]);
    }
    // Ey at (i, j+1/2, k): D-_z Hx - D-_x Hz
    if (FAST || (j <= np1 - 2 && dm_i && dm_k)) {
      float dz = 0.f, dx = 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        dz = fmaf(cz[q], v.zf(c + q, ty + R, tx), dz);
        dx = fmaf(cx[q], v.xy(c, ty + R, tx + XH - R + q), dx);
      }
      if (!FAST) {
        if (sk >= 0)
          dz = cpml_step(dz, ps[(2 * ZC + c) * NT + threadIdx.x], p.psiE[2], psi_at(2, sk, i, j, k, p.np, 2 * nb),
                         p.pml[2][sk], p.pml[2][2 * nb + sk]);
        if (si >= 0)
          dx = cpml_step(dx, ps[(3 * ZC + c) * NT + threadIdx.x], p.psiE[3], psi_at(0, si, i, j, k, p.np, 2 * nb),
                         p.pml[0][si], p.pml[0][2 * nb + si]);
      }
      float curl = dz - dx;
      if (!FAST && src) source_term<R>(p, 1, i, j, k, amp, curl);
      p.E[1][id] = fmaf(w[1][c], curl, e[1][c]);
    }
    // Ez at (i, j, k+1/2): D-_x Hy - D-_y Hx
    if (FAST || (dm_i && dm_j && k <= np2 - 2)) {
      float dx = 0.f, dy = 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        dx = fmaf(cx[q], v.xf(c + R, ty, tx + XH - R + q), dx);
        dy = fmaf(cy[q], v.zf(c + R, ty + q, tx), dy);
      }
      if (!FAST) {
        if (si >= 0)
          dx = cpml_step(dx, ps[(4 * ZC + c) * NT + threadIdx.x], p.psiE[4], psi_at(0, si, i, j, k, p.np, 2 * nb),
                         p.pml[0][si], p.pml[0][2 * nb + si]);
        if (sj >= 0)
          dy = cpml_step(dy, ps[(5 * ZC + c) * NT + threadIdx.x], p.psiE[5], psi_at(1, sj, i, j, k, p.np, 2 * nb),
                         p.pml[1][sj], p.pml[1][2 * nb + sj]);
      }
      float curl = dx - dy;
      if (!FAST && src) source_term<R>(p, 2, i, j, k, amp, curl);
      p.E[2][id] = fmaf(w[2][c], curl, e[2][c]);
    }
    // volume DTFT of H^{n+1/2}
    if (VOL) {
      const int kk = k - p.nbe;
      if (int_ij && kk >= 0 && kk < p.n[2]) {
        const int lin = (kk * p.n[1] + jj) * p.n[0] + ii;
        volume_accumulate(p, 3, lin, nint, facH, v.zf(c + R, ty + R, tx));
        volume_accumulate(p, 4, lin, nint, facH, v.xf(c + R, ty, tx + XH));
        volume_accumulate(p, 5, lin, nint, facH, v.xy(c, ty + R, tx + XH));
      }
    }
  }
}

template <int R, bool VOL>
__global__ void __launch_bounds__(NT, min_ctas(R))
    k_update_E(const DevParams p, const __grid_constant__ TmaSet tm, const int n) {
  if (static_cast<int>(blockIdx.x) >= p.stencil_blocks) {
    receiver_dft<R>(p, 3, p.H, p.fH + static_cast<size_t>(n) * p.nf * 2, blockIdx.x - p.stencil_blocks);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  float *s = smem_tiles(smem_raw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(s + Tiles<R>::ALL / 4);
  const Origin o = origin_of(p, blockIdx.x);
  if (threadIdx.x == 0) issue_tiles<R>(tm, s, bar, o, -R);

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = o.i0 + tx, j = o.j0 + ty;
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const bool in_ij = i >= 0 && i < np0 && j >= 0 && j < np1;
  const size_t col = static_cast<size_t>(j) * p.pitch + i;
  // this thread's own samples, loaded while the copies are in flight
  float e[3][ZC], w[3][ZC];
#pragma unroll
  for (int c = 0; c < ZC; ++c) {
    const int k = o.k0 + c;
    const bool ok = in_ij && k >= 0 && k < np2;
    const size_t id = static_cast<size_t>(k) * p.plane + col;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      e[a][c] = ok ? p.E[a][id] : 0.f;
      w[a][c] = ok ? __ldg(p.ie[a] + id) : 0.f;
    }
  }
  const bool src = cta_has_source(p, o);
  const bool fast = !src && interior_E(p, o, R);
  float *ps = s + Tiles<R>::BYTES / 4;
  if (!fast && in_ij)
    stage_psi(ps, p.psiE, p, i, j, o.k0, slab_int(i, np0, nb), slab_int(j, np1, nb),
              [&](int k) { return slab_int(k, np2, nb); });
  else
    cp_async_commit();
  cp_async_wait_all();
  if (!tiles_ready(p, bar) || !in_ij) return;
  const View<R> v{s};
  if (fast)
    e_planes<R, VOL, true>(p, v, o, tx, ty, e, w, ps, n, false);
  else
    e_planes<R, VOL, false>(p, v, o, tx, ty, e, w, ps, n, src);
}

// ---------------------------------------------------------------------------
// H half-step: H^{n+3/2} = H^{n+1/2} - dt/mu0 curl E^{n+1}
// ---------------------------------------------------------------------------
// Is every cell of the CTA inside the CPML-free region where all D+ rows exist?
__device__ __forceinline__ bool interior_H(const DevParams &p, const Origin &o, int R) {
  const int lo = max(p.nb, R - 1);
  const int hx = min(p.np[0] - 2 - p.nb, p.np[0] - 1 - R), hy = min(p.np[1] - 2 - p.nb, p.np[1] - 1 - R),
            hz = min(p.np[2] - 2 - p.nb, p.np[2] - 1 - R);
  return o.i0 >= lo && o.i0 + TX - 1 <= hx && o.j0 >= lo && o.j0 + TY - 1 <= hy && o.k0 >= lo &&
         o.k0 + ZC - 1 <= hz;
}

template <int R, bool VOL, bool FAST>
__device__ __forceinline__ void h_planes(const DevParams &p, const View<R> &v, const Origin &o, int tx, int ty,
                                         const float (&h)[3][ZC], const float *ps, int n) {
  constexpr int M = 2 * R;
  const int i = o.i0 + tx, j = o.j0 + ty;
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const size_t col = static_cast<size_t>(j) * p.pitch + i;
  const bool dp_i = FAST || (i >= R - 1 && i <= np0 - 1 - R), dp_j = FAST || (j >= R - 1 && j <= np1 - 1 - R);
  const int si = FAST ? -1 : slab_half(i, np0, nb), sj = FAST ? -1 : slab_half(j, np1, nb);
  float cx[M], cy[M];
#pragma unroll
  for (int q = 0; q < M; ++q) {
    cx[q] = dp_i ? __ldg(p.cp[0] + i * M + q) : 0.f;
    cy[q] = dp_j ? __ldg(p.cp[1] + j * M + q) : 0.f;
  }
  const float dt_mu = p.dt_mu;
  const int ii = i - p.nbe, jj = j - p.nbe;
  const bool int_ij = VOL && ii >= 0 && ii < p.n[0] && jj >= 0 && jj < p.n[1];
  const size_t nint = static_cast<size_t>(p.n[0]) * p.n[1] * p.n[2];
  const float *facE = p.fE32 + static_cast<size_t>(n) * p.nf * 2;

#pragma unroll
  for (int c = 0; c < ZC; ++c) {
    const int k = o.k0 + c;
    if (!FAST) {
      if (k < 0) continue;
      if (k >= np2) break;
    }
    const size_t id = static_cast<size_t>(k) * p.plane + col;
    const bool dp_k = FAST || (k >= R - 1 && k <= np2 - 1 - R);
    const int sk = FAST ? -1 : slab_half(k, np2, nb);
    float cz[M];
#pragma unroll
    for (int q = 0; q < M; ++q) cz[q] = dp_k ? __ldg(p.cp[2] + k * M + q) : 0.f;
    // Hx at (i, j+1/2, k+1/2): D+_y Ez - D+_z Ey
    if (FAST || (dp_j && dp_k)) {
      float dy = 0.f, dz = 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        dy = fmaf(cy[q], v.xy(c, ty + q + 1, tx + XH), dy);
        dz = fmaf(cz[q], v.xf(c + q, ty, tx + XH), dz);
      }
      if (!FAST) {
        if (sj >= 0)
          dy = cpml_step(dy, ps[(0 * ZC + c) * NT + threadIdx.x], p.psiH[0], psi_at(1, sj, i, j, k, p.np, 2 * nb),
                         p.pml[1][4 * nb + sj], p.pml[1][6 * nb + sj]);
        if (sk >= 0)
          dz = cpml_step(dz, ps[(1 * ZC + c) * NT + threadIdx.x], p.psiH[1], psi_at(2, sk, i, j, k, p.np, 2 * nb),
                         p.pml[2][4 * nb + sk], p.pml[2][6 * nb + sk]);
      }
      p.H[0][id] = fmaf(-dt_mu, dy - dz, h[0][c]);
    }
    // Hy at (i+1/2, j, k+1/2): D+_z Ex - D+_x Ez
    if (FAST || (dp_i && dp_k)) {
      float dz = 0.f, dx = 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        dz = fmaf(cz[q], v.zf(c + q, ty + R, tx), dz);
        dx = fmaf(cx[q], v.xy(c, ty + R, tx + XH - R + 1 + q), dx);
      }
      if (!FAST) {
        if (sk >= 0)
          dz = cpml_step(dz, ps[(2 * ZC + c) * NT + threadIdx.x], p.psiH[2], psi_at(2, sk, i, j, k, p.np, 2 * nb),
                         p.pml[2][4 * nb + sk], p.pml[2][6 * nb + sk]);
        if (si >= 0)
          dx = cpml_step(dx, ps[(3 * ZC + c) * NT + threadIdx.x], p.psiH[3], psi_at(0, si, i, j, k, p.np, 2 * nb),
                         p.pml[0][4 * nb + si], p.pml[0][6 * nb + si]);
      }
      p.H[1][id] = fmaf(-dt_mu, dz - dx, h[1][c]);
    }
    // Hz at (i+1/2, j+1/2, k): D+_x Ey - D+_y Ex
    if (FAST || (dp_i && dp_j)) {
      float dx = 0.f, dy = 0.f;
#pragma unroll
      for (int q = 0; q < M; ++q) {
        dx = fmaf(cx[q], v.xf(c + R - 1, ty, tx + XH - R + 1 + q), dx);
        dy = fmaf(cy[q], v.zf(c + R - 1, ty + q + 1, tx), dy);
      }
      if (!FAST) {
        if (si >= 0)
          dx = cpml_step(dx, ps[(4 * ZC + c) * NT + threadIdx.x], p.psiH[4], psi_at(0, si, i, j, k, p.np, 2 * nb),
                         p.pml[0][4 * nb + si], p.pml[0][6 * nb + si]);
        if (sj >= 0)
          dy = cpml_step(dy, ps[(5 * ZC + c) * NT + threadIdx.x], p.psiH[5], psi_at(1, sj, i, j, k, p.np, 2 * nb),
                         p.pml[1][4 * nb + sj], p.pml[1][6 * nb + sj]);
      }
      p.H[2][id] = fmaf(-dt_mu, dx - dy, h[2][c]);
    }
    // volume DTFT of E^{n+1}
    if (VOL) {
      const int kk = k - p.nbe;
      if (int_ij && kk >= 0 && kk < p.n[2]) {
        const int lin = (kk * p.n[1] + jj) * p.n[0] + ii;
        volume_accumulate(p, 0, lin, nint, facE, v.zf(c + R - 1, ty + R, tx));
        volume_accumulate(p, 1, lin, nint, facE, v.xf(c + R - 1, ty, tx + XH));
        volume_accumulate(p, 2, lin, nint, facE, v.xy(c, ty + R, tx + XH));
      }
    }
  }
}

template <int R, bool VOL>
__global__ void __launch_bounds__(NT, min_ctas(R))
    k_update_H(const DevParams p, const __grid_constant__ TmaSet tm, const int n) {
  if (static_cast<int>(blockIdx.x) >= p.stencil_blocks) {
    receiver_dft<R>(p, 0, p.E, p.fE + static_cast<size_t>(n) * p.nf * 2, blockIdx.x - p.stencil_blocks);
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  float *s = smem_tiles(smem_raw);
  uint64_t *bar = reinterpret_cast<uint64_t *>(s + Tiles<R>::ALL / 4);
  const Origin o = origin_of(p, blockIdx.x);
  if (threadIdx.x == 0) issue_tiles<R>(tm, s, bar, o, 1 - R);

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = o.i0 + tx, j = o.j0 + ty;
  const int np0 = p.np[0], np1 = p.np[1], np2 = p.np[2], nb = p.nb;
  const bool in_ij = i >= 0 && i < np0 && j >= 0 && j < np1;
  const size_t col = static_cast<size_t>(j) * p.pitch + i;
  float h[3][ZC];
#pragma unroll
  for (int c = 0; c < ZC; ++c) {
    const int k = o.k0 + c;
    const bool ok = in_ij && k >= 0 && k < np2;
    const size_t id = static_cast<size_t>(k) * p.plane + col;
#pragma unroll
    for (int a = 0; a < 3; ++a) h[a][c] = ok ? p.H[a][id] : 0.f;
  }
  const bool fast = interior_H(p, o, R);
  float *ps = s + Tiles<R>::BYTES / 4;
  if (!fast && in_ij)
    stage_psi(ps, p.psiH, p, i, j, o.k0, slab_half(i, np0, nb), slab_half(j, np1, nb),
              [&](int k) { return slab_half(k, np2, nb); });
  else
    cp_async_commit();
  cp_async_wait_all();
  if (!tiles_ready(p, bar) || !in_ij) return;
  const View<R> v{s};
  if (fast)
    h_planes<R, VOL, true>(p, v, o, tx, ty, h, ps, n);
  else
    h_planes<R, VOL, false>(p, v, o, tx, ty, h, ps, n);
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

// ---------------------------------------------------------------------------
// Host side of emm_forward
// ---------------------------------------------------------------------------
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
};
FieldGeom field_geom(const emm_grid *g) {
  FieldGeom f{};
  const int lo = std::max(g->nb, g->rd);
  const int lo4 = lo & ~3;
  const int step[3] = {TX, TY, ZC};
  const int first[3] = {lo4, lo, lo};
  for (int a = 0; a < 3; ++a) {
    f.org[a] = first[a] - step[a] * ((first[a] + step[a] - 1) / step[a]);
    f.tiles[a] = (g->ax[a].npad - f.org[a] + step[a] - 1) / step[a];
  }
  f.xshift = -f.org[0];
  f.pitch = (g->ax[0].npad + f.xshift + 31) / 32 * 32;
  return f;
}

// Byte layout of the device workspace.
struct Layout {
  size_t status, E[3], H[3], ie[3], psiE[6], psiH[6], vacc, zero_end;
  size_t cm[3], cp[3], pml[3], jw[3], amp, rec_start, rec_w, fE, fH, fE32, fH32, norm, total;
};

size_t psi_elems(const emm_grid *g, int axis) {
  const size_t nb2 = 2 * static_cast<size_t>(g->nb);
  const size_t p0 = g->ax[0].npad, p1 = g->ax[1].npad, p2 = g->ax[2].npad;
  if (axis == 0) return p2 * p1 * nb2;
  if (axis == 1) return p2 * nb2 * p0;
  return nb2 * p1 * p0;
}

// Derivative axis of CPML array c (0..5): 2*comp + 0 -> (comp+1)%3, 2*comp + 1 -> (comp+2)%3.
inline int psi_axis(int c) { return (c % 2 == 0) ? (c / 2 + 1) % 3 : (c / 2 + 2) % 3; }

Layout plan(const emm_grid *g, const emm_survey *s) {
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
  for (int c = 0; c < 3; ++c) L.E[c] = take(cells * 4);
  for (int c = 0; c < 3; ++c) L.H[c] = take(cells * 4);
  for (int c = 0; c < 6; ++c) L.psiE[c] = take(psi_elems(g, psi_axis(c)) * 4);
  for (int c = 0; c < 6; ++c) L.psiH[c] = take(psi_elems(g, psi_axis(c)) * 4);
  L.vacc = take(s->volume ? 6 * nf * nint * sizeof(float4) : 0);
  L.zero_end = off;
  for (int c = 0; c < 3; ++c) L.ie[c] = take(cells * 4);
  for (int a = 0; a < 3; ++a) L.cm[a] = take(static_cast<size_t>(g->ax[a].npad) * m * 4);
  for (int a = 0; a < 3; ++a) L.cp[a] = take(static_cast<size_t>(g->ax[a].npad) * m * 4);
  for (int a = 0; a < 3; ++a) L.pml[a] = take(8 * static_cast<size_t>(g->nb) * 4);
  for (int c = 0; c < 3; ++c) L.jw[c] = take(m * m * m * 4);
  L.amp = take(nt * 4);
  L.rec_start = take(nrec * 18 * sizeof(int));
  L.rec_w = take(nrec * 18 * m * sizeof(double));
  L.fE = take(nt * nf * 2 * sizeof(double));
  L.fH = take(nt * nf * 2 * sizeof(double));
  L.fE32 = take(nt * nf * 2 * sizeof(float));
  L.fH32 = take(nt * nf * 2 * sizeof(float));
  L.norm = take(2 * nf * 2 * sizeof(double));
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
  return EMM_OK;
}

// cuTensorMapEncodeTiled, fetched once from the driver through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

// 3-D FP32 tensor [np2][np1][pitch] (dims np0 x np1 x np2), box bx x by x bz.
bool make_map(CUtensorMap *map, const float *base, const DevParams &p, int bx, int by, int bz) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(p.np[0]), static_cast<cuuint64_t>(p.np[1]),
                              static_cast<cuuint64_t>(p.np[2])};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(p.pitch) * 4, static_cast<cuuint64_t>(p.plane) * 4};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(bx), static_cast<cuuint32_t>(by),
                             static_cast<cuuint32_t>(bz)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The boxes of the three source fields (see Tiles).
template <int R>
bool make_tiles(TmaSet *t, float *const *F, const DevParams &p) {
  using T = Tiles<R>;
  return make_map(&t->m[0], F[0], p, TX, T::YH, T::ZQ) && make_map(&t->m[1], F[1], p, WX, TY, T::ZQ) &&
         make_map(&t->m[2], F[2], p, WX, T::YH, ZC);
}

// Optional per-launch timing: events before/after the E and H launches of
// every `every`-th step (3 events per timed step).
struct StepEvents {
  int every = 0;
  std::vector<cudaEvent_t> ev;
};

template <int R, bool VOL>
cudaError_t launch_steps(const DevParams &p, int nt, int blocks, cudaStream_t st, StepEvents *te) {
  TmaSet tE{}, tH{};
  if (!make_tiles<R>(&tE, p.H, p) || !make_tiles<R>(&tH, p.E, p)) return cudaErrorInvalidValue;
  const size_t sb = smem_bytes<R>();
  cudaError_t e =
      cudaFuncSetAttribute(k_update_E<R, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sb));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_update_H<R, VOL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sb));
  if (e != cudaSuccess) return e;
  size_t used = 0;
  for (int n = 0; n < nt; ++n) {
    const bool timed = te && te->every > 0 && (n % te->every) == 0 && used + 3 <= te->ev.size();
    if (timed) cudaEventRecord(te->ev[used], st);
    k_update_E<R, VOL><<<blocks, NT, sb, st>>>(p, tE, n);
    if (timed) cudaEventRecord(te->ev[used + 1], st);
    k_update_H<R, VOL><<<blocks, NT, sb, st>>>(p, tH, n);
    if (timed) {
      cudaEventRecord(te->ev[used + 2], st);
      used += 3;
    }
  }
  return cudaGetLastError();
}

int forward_impl(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                 double *rec_out, double *vol_out, emm_stream stream, StepEvents *te) {
  int st = check_survey(g, s);
  if (st != EMM_OK) return st;
  if (!sigma || !ws || (s->nrec > 0 && !rec_out) || (s->volume && !vol_out)) return EMM_EINVAL;
  const Layout L = plan(g, s);
  if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return EMM_EWORKSPACE;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
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
    float *pm = reinterpret_cast<float *>(at(L.pml[a]));
    for (size_t q = 0; q < ab.size(); ++q) pm[q] = static_cast<float>(ab[q]);
  }
  // source: J_node = moment s(t) dir_c w_node / V_node, V = dual-cell volume
  const double dir[3] = {std::cos(s->src_dip) * std::cos(s->src_az), std::cos(s->src_dip) * std::sin(s->src_az),
                         std::sin(s->src_dip)};
  DevParams p{};
  for (int c = 0; c < 3; ++c) {
    p.src_on[c] = 0;
    if (dir[c] == 0.0) continue;
    int start[3];
    double w[3][2 * kMaxRd];
    for (int a = 0; a < 3; ++a) {
      st = locate_axis(g, a, kHalf[c][a], s->src[a], &start[a], w[a]);
      if (st != EMM_OK) return st;
    }
    float *jw = reinterpret_cast<float *>(at(L.jw[c]));
    for (int q3 = 0; q3 < m; ++q3)
      for (int q2 = 0; q2 < m; ++q2)
        for (int q1 = 0; q1 < m; ++q1) {
          const int idx[3] = {start[0] + q1, start[1] + q2, start[2] + q3};
          double vol = 1.0;
          for (int a = 0; a < 3; ++a) {
            const Axis &ax = g->ax[a];
            vol *= kHalf[c][a] ? (ax.X[idx[a] + 1] - ax.X[idx[a]]) : (ax.Xh[idx[a]] - ax.Xh[idx[a] - 1]);
          }
          jw[(q3 * m + q2) * m + q1] = static_cast<float>(dir[c] * w[0][q1] * w[1][q2] * w[2][q3] / vol);
        }
    p.src_on[c] = 1;
    for (int a = 0; a < 3; ++a) p.src_start[c][a] = start[a];
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
  std::vector<std::complex<double>> jhat(nf, 0.0), wp(nf);
  for (int f = 0; f < nf; ++f)
    wp[f] = std::complex<double>(1.0, 1.0) * std::sqrt(2.0 * M_PI * s->freqs[f] * s->omega0);
  const double t0 = 1.5 / s->fmax;
  const std::complex<double> I(0.0, 1.0);
  for (int n = 0; n < nt; ++n) {
    const double th = (n + 0.5) * dt, te_ = (n + 1.0) * dt;
    const double u = M_PI * s->fmax * (th - t0);
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
      jhat[f] += eH * a;  // J is sampled at t_{n+1/2}, the H label
    }
  }
  // normalisation (Eq. 7): G^EE = sqrt(-i w / (2 w0)) E'/J', G^HE = H'/J'
  double *norm = reinterpret_cast<double *>(at(L.norm));
  for (int f = 0; f < nf; ++f) {
    const std::complex<double> sE =
        std::sqrt(2.0 * M_PI * s->freqs[f] / (2.0 * s->omega0)) * std::exp(-I * (M_PI / 4.0));
    const std::complex<double> nE = (jhat[f] != 0.0) ? sE / jhat[f] : 0.0;
    const std::complex<double> nH = (jhat[f] != 0.0) ? 1.0 / jhat[f] : 0.0;
    norm[2 * f] = nE.real();
    norm[2 * f + 1] = nE.imag();
    norm[2 * nf + 2 * f] = nH.real();
    norm[2 * nf + 2 * f + 1] = nH.imag();
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
  const FieldGeom fg = field_geom(g);
  p.pitch = fg.pitch;
  p.plane = static_cast<size_t>(p.pitch) * p.np[1];
  p.nbe = nbe;
  p.nb = nb;
  for (int c = 0; c < 3; ++c) {
    p.E[c] = reinterpret_cast<float *>(base + L.E[c]) + fg.xshift;
    p.H[c] = reinterpret_cast<float *>(base + L.H[c]) + fg.xshift;
    p.ie[c] = reinterpret_cast<const float *>(base + L.ie[c]) + fg.xshift;
    p.jw[c] = reinterpret_cast<const float *>(base + L.jw[c]);
  }
  for (int c = 0; c < 6; ++c) {
    p.psiE[c] = reinterpret_cast<float *>(base + L.psiE[c]);
    p.psiH[c] = reinterpret_cast<float *>(base + L.psiH[c]);
  }
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
  p.rec_blocks = (s->nrec * 3 + NT / 32 - 1) / (NT / 32);
  const int blocks = p.stencil_blocks + p.rec_blocks;
  // bounding box of the source stencils (lets CTAs far from it skip the test)
  p.src_any = 0;
  for (int a = 0; a < 3; ++a) {
    p.src_lo[a] = 1 << 30;
    p.src_hi[a] = -1;
  }
  for (int c = 0; c < 3; ++c)
    if (p.src_on[c]) {
      p.src_any = 1;
      for (int a = 0; a < 3; ++a) {
        p.src_lo[a] = std::min(p.src_lo[a], p.src_start[c][a]);
        p.src_hi[a] = std::max(p.src_hi[a], p.src_start[c][a] + m - 1);
      }
    }

  // ---- enqueue ----
  cudaError_t e = cudaMemsetAsync(ws, 0, L.zero_end, cs);
  if (e == cudaSuccess && s->nrec > 0)
    e = cudaMemsetAsync(rec_out, 0, static_cast<size_t>(s->nrec) * 6 * nf * 2 * sizeof(double), cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + tab0, blob.data(), blob.size(), cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return EMM_ECUDA;
  k_prepare<<<4 * sms, 256, 0, cs>>>(sigma, reinterpret_cast<float *>(base + L.ie[0]),
                                     reinterpret_cast<float *>(base + L.ie[1]),
                                     reinterpret_cast<float *>(base + L.ie[2]), p.n[0], p.n[1], p.n[2], p.np[0],
                                     p.np[1], p.np[2], p.pitch, fg.xshift, nbe, 2.0 * s->omega0 * dt, s->sigma_min,
                                     p.status);
  const bool vol = p.vacc != nullptr;
  switch (rd) {
    case 1: e = vol ? launch_steps<1, true>(p, nt, blocks, cs, te) : launch_steps<1, false>(p, nt, blocks, cs, te);
      break;
    case 2: e = vol ? launch_steps<2, true>(p, nt, blocks, cs, te) : launch_steps<2, false>(p, nt, blocks, cs, te);
      break;
    case 3: e = vol ? launch_steps<3, true>(p, nt, blocks, cs, te) : launch_steps<3, false>(p, nt, blocks, cs, te);
      break;
    default: e = vol ? launch_steps<4, true>(p, nt, blocks, cs, te) : launch_steps<4, false>(p, nt, blocks, cs, te);
      break;
  }
  if (e != cudaSuccess) return EMM_ECUDA;
  const double *dnorm = reinterpret_cast<const double *>(base + L.norm);
  if (s->nrec > 0) {
    const int tot = s->nrec * 6 * nf;
    k_finalize_rec<<<(tot + 255) / 256, 256, 0, cs>>>(rec_out, dnorm, s->nrec, nf);
  }
  if (s->volume) {
    const size_t nint = static_cast<size_t>(p.n[0]) * p.n[1] * p.n[2];
    k_finalize_vol<<<8 * sms, 256, 0, cs>>>(p.vacc, vol_out, dnorm, nint, nf);
  }
  return cudaGetLastError() == cudaSuccess ? EMM_OK : EMM_ECUDA;
}

// Device address of emm_static_scratch on the current device, looked up once
// per device (with that device current) and cached.
int static_scratch(void **ptr) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static void *addr[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return EMM_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (dev < kMaxDevices && addr[dev]) {
    *ptr = addr[dev];
    return EMM_OK;
  }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, emm_static_scratch) != cudaSuccess || !p) return EMM_ECUDA;
  if (dev < kMaxDevices) addr[dev] = p;
  *ptr = p;
  return EMM_OK;
}

}  // namespace
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
  std::vector<cudaEvent_t> all(3 * static_cast<size_t>(nsamp) + 2, nullptr);
  for (auto &e : all)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto &d : all)
        if (d) cudaEventDestroy(d);
      return EMM_ECUDA;
    }
  StepEvents te;
  te.every = timing->every;
  te.ev.assign(all.begin(), all.begin() + 3 * static_cast<size_t>(nsamp));
  cudaEvent_t t0 = all[all.size() - 2], t1 = all[all.size() - 1];
  cudaEventRecord(t0, cs);
  st = forward_impl(g, s, sigma, ws, ws_bytes, rec_out, vol_out, stream, &te);
  cudaEventRecord(t1, cs);
  if (cudaStreamSynchronize(cs) != cudaSuccess && st == EMM_OK) st = EMM_ECUDA;
  double se = 0, sh = 0;
  float ms = 0.f;
  for (int q = 0; q < nsamp && st == EMM_OK; ++q) {
    cudaEventElapsedTime(&ms, te.ev[3 * q], te.ev[3 * q + 1]);
    se += ms;
    cudaEventElapsedTime(&ms, te.ev[3 * q + 1], te.ev[3 * q + 2]);
    sh += ms;
  }
  timing->samples = nsamp;
  timing->e_ms = nsamp ? se / nsamp : 0.0;
  timing->h_ms = nsamp ? sh / nsamp : 0.0;
  ms = 0.f;
  if (st == EMM_OK) cudaEventElapsedTime(&ms, t0, t1);
  timing->total_ms = ms;
  for (auto &e : all) cudaEventDestroy(e);
  return st;
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
