// VGICP factor linearization kernels (arXiv 2202.00242 Sec. III-A, Eqs. 2-3 and
// the Hessian factor built from their derivatives at every optimizer iteration).
//
// One persistent launch processes a list of work items (pair, [begin, end)) over
// the source clouds.  Per source point k of pair (map, source, T = (R, t)):
//   q    = R mu_k + t                                   (float32)
//   key  = floor(q / r) exactly as in binary64 (float32 fast path, binary64
//          recomputation for the rare points whose float32 q lies within its
//          error bound of a voxel face)
//   vid  = hash lookup (open addressing, bounded linear probe)
//   in the SOURCE frame (J = R K with K = [[mu]x, -I], so J^T W J = K^T W' K):
//   d'   = R^T (mu'_v - q)
//   M'   = R^T C'_v R + C_k = B B^T + C_k with B = R^T L (C'_v = L L^T, the
//          Cholesky factor kept in the lookup slot), W' = M'^-1 (= R^T W R,
//          symmetric adjugate / det)
//   u    = W' d'
//   err += d'^T u
//   b   += [ u x mu ; -u ]
//   H   += [[ [mu]x^T W' [mu]x , [mu]x W' ], [ ., W' ]]
// The 28 unique terms and the inlier count are accumulated per thread in
// float32 over a work item (up to 16K points of one pair), reduced across the
// warp in float32, across warps in binary64, and written as one binary64
// partial per work item; a second kernel sums each pair's partials in item
// order.  The result is deterministic.
//
// Work items are claimed dynamically from an atomic counter, so uneven items
// (ragged tails of the clouds, pairs with few inliers) do not leave CTAs idle.
//
// Kernels (the autotuner picks among the 1-neighbour ones per factor set):
//   1  per-point: one point per thread, item constants in shared memory so that
//      3 CTAs of 256 threads fit per SM; the default and usually the fastest;
//   2  staged: a producer warp streams tiles of points and covariances into
//      shared memory with bulk asynchronous copies (cp.async.bulk + mbarrier);
//      consumer warps look up, compact the hits and evaluate from shared memory;
//   3  compacting: the per-point lookup, with the hits queued per warp in shared
//      memory and evaluated 32 at a time (no idle lanes on misses);
//   27 neighbours: the per-point kernel with the 27 lookups in a loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "vgicp_device.cuh"
#include "vgicp_internal.h"

namespace vgicp {
namespace {

constexpr int kSimpleThreads = 256;

struct Pose32 {
  float R[9];
  float t[3];
  float tmax;
};

// floor(q_a / r) with q = R64 mu + t64 in binary64 (the rare near-face path).
__device__ __noinline__ int axis_key_f64(const PairDesc* pd, const MapDesc& md, int a, float x,
                                         float y, float z) {
  double s = __dmul_rn(pd->R64[3 * a + 0], (double)x);
  s = __dadd_rn(s, __dmul_rn(pd->R64[3 * a + 1], (double)y));
  s = __dadd_rn(s, __dmul_rn(pd->R64[3 * a + 2], (double)z));
  s = __dadd_rn(s, pd->t64[a]);
  double k = floor(__ddiv_rn(s, md.r));
  k = fmin(fmax(k, -2147483648.0), 2147483647.0);
  return (int)k;
}

// Key of the transformed source point, exact w.r.t. the binary64 definition
// floor((R64 mu + t64) / r).  Float32 bound: |q32 - q64| <= 2^-22 S with
// S = |x| + |y| + |z| + max|t| (rounding of R and t to float32 and three FMA
// roundings), and y = q32 * float(1/r) adds 2^-23 |y|; the margin
// 2^-21 S / r + 2^-23 covers both and the rounding of the fractional part.
__device__ __forceinline__ void source_key(const Pose32& P, const PairDesc* pd, const MapDesc& md,
                                           float x, float y, float z, float qx, float qy,
                                           float qz, int& kx, int& ky, int& kz) {
  const float S = fabsf(x) + fabsf(y) + fabsf(z) + P.tmax;
  const float m = fmaf(S, md.margin_scale, 1.1920928955078125e-7f);
  const float yx = qx * md.inv_r, yy = qy * md.inv_r, yz = qz * md.inv_r;
  const float fx = floorf(yx), fy = floorf(yy), fz = floorf(yz);
  const float rx = yx - fx, ry = yy - fy, rz = yz - fz;
  const bool ax = (rx < m) | (rx > 1.0f - m);
  const bool ay = (ry < m) | (ry > 1.0f - m);
  const bool az = (rz < m) | (rz > 1.0f - m);
  kx = clamp_to_int(fx);
  ky = clamp_to_int(fy);
  kz = clamp_to_int(fz);
  if (ax | ay | az) {
    // binary64, evaluated as ((R0 x + R1 y) + R2 z) + t without contraction
    if (ax) kx = axis_key_f64(pd, md, 0, x, y, z);
    if (ay) ky = axis_key_f64(pd, md, 1, x, y, z);
    if (az) kz = axis_key_f64(pd, md, 2, x, y, z);
  }
}

// Two independent 256-bit loads: one probe of a 64-B lookup slot.
#ifndef VGICP_LD_FLAVOR
#define VGICP_LD_FLAVOR 0
#endif
__device__ __forceinline__ void ld_v8(const void* p, uint64_t policy, uint32_t (&w)[8]) {
#if VGICP_LD_FLAVOR == 0
  asm("ld.global.nc.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
        "=r"(w[7])
      : "l"(p), "l"(policy));
#elif VGICP_LD_FLAVOR == 1
  asm("ld.global.cg.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
        "=r"(w[7])
      : "l"(p), "l"(policy));
#else
  asm("ld.global.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
        "=r"(w[7])
      : "l"(p), "l"(policy));
#endif
}
__device__ __forceinline__ unsigned long long slot_key(const uint32_t (&a)[8]) {
  return (unsigned long long)a[0] | ((unsigned long long)a[1] << 32);
}
// A slot's first 16 B: key (words 0, 1), spill flag, vid.
__device__ __forceinline__ void ld_v4(const void* p, uint64_t policy, uint32_t (&w)[4]) {
  asm("ld.global.nc.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
      : "l"(p), "l"(policy));
}
__device__ __forceinline__ uint64_t policy_evict_last_l() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Lookup of key (kx, ky, kz) in a map's inline table; on a hit returns the
// global voxel id and the voxel Gaussian as r0 = (mu', -), r1, r2 (record layout).
__device__ __forceinline__ int lookup(const MapDesc& md, uint32_t mask, int kx, int ky, int kz,
                                      uint64_t pol, float4& r0, float4& r1, float4& r2) {
  if (!key_in_range(kx) || !key_in_range(ky) || !key_in_range(kz)) return -1;
  const unsigned long long key = pack_key(kx, ky, kz);
  uint32_t h = hash_key(kx, ky, kz) & mask;
  for (int p = 0; p < md.max_probe; ++p) {
    uint32_t a[8], b[8];
    const VSlot* t = md.vslots + h;
    ld_v8(t, pol, a);
    ld_v8(reinterpret_cast<const char*>(t) + 32, pol, b);
    const unsigned long long k = slot_key(a);
    if (k == key) {
      r0 = make_float4(__uint_as_float(a[kSlotMu]), __uint_as_float(a[kSlotMu + 1]),
                       __uint_as_float(a[kSlotMu + 2]), 0.f);
      r1 = make_float4(__uint_as_float(b[0]), __uint_as_float(b[1]), __uint_as_float(b[2]),
                       __uint_as_float(b[3]));
      r2 = make_float4(__uint_as_float(b[4]), __uint_as_float(b[5]), 0.f, 0.f);
      return (int)a[kSlotVid];
    }
    if (k == kEmptyKey || (p == 0 && a[kSlotSpill] == 0u)) return -1;  // empty, or nothing spilled
    h = (h + 1) & mask;
  }
  return -1;
}

// Accumulator layout (float):
//   0..5   H_ww (00 01 02 11 12 22)      6..14 H_wv (row-major, w rows, v cols)
//   15..20 H_vv (00 01 02 11 12 22)      21..23 b_w   24..26 b_v   27 err
//   28     inlier count
// 1 / x to about 1 ulp (rcp.approx: one instruction; H, b and err are held to
// 1e-4 relative, many orders above this).  Deterministic.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// M' = R^T C' R + C (upper triangle m00 m01 m02 m11 m12 m22) from the voxel
// covariance's Cholesky factor L (C' = L L^T, stored in the lookup slot as
// l00 l10 l20 l11 l21 l22): with B = R^T L, R^T C' R = B B^T (36 operations
// instead of 45 for R^T (C' R)).
__device__ __forceinline__ void fused_cov(const float* R, const float4 r1, const float4 r2,
                                          const float* c, float& m00, float& m01, float& m02,
                                          float& m11, float& m12, float& m22) {
  const float l00 = r1.x, l10 = r1.y, l20 = r1.z, l11 = r1.w, l21 = r2.x, l22 = r2.y;
  // B_i0 = sum_k R_ki L_k0, B_i1 = R_1i l11 + R_2i l21, B_i2 = R_2i l22
  const float b00 = fmaf(R[0], l00, fmaf(R[3], l10, R[6] * l20));
  const float b10 = fmaf(R[1], l00, fmaf(R[4], l10, R[7] * l20));
  const float b20 = fmaf(R[2], l00, fmaf(R[5], l10, R[8] * l20));
  const float b01 = fmaf(R[3], l11, R[6] * l21);
  const float b11 = fmaf(R[4], l11, R[7] * l21);
  const float b21 = fmaf(R[5], l11, R[8] * l21);
  const float b02 = R[6] * l22, b12 = R[7] * l22, b22 = R[8] * l22;
  m00 = fmaf(b00, b00, fmaf(b01, b01, fmaf(b02, b02, c[0])));
  m01 = fmaf(b00, b10, fmaf(b01, b11, fmaf(b02, b12, c[1])));
  m02 = fmaf(b00, b20, fmaf(b01, b21, fmaf(b02, b22, c[2])));
  m11 = fmaf(b10, b10, fmaf(b11, b11, fmaf(b12, b12, c[3])));
  m12 = fmaf(b10, b20, fmaf(b11, b21, fmaf(b12, b22, c[4])));
  m22 = fmaf(b20, b20, fmaf(b21, b21, fmaf(b22, b22, c[5])));
}

__device__ __forceinline__ void add_term_t(float* acc, const float* R, float x, float y, float z,
                                           const float* c, float tx, float ty, float tz,
                                           const float4 r1, const float4 r2) {
  // residual (tx, ty, tz) = mu' - q in the target frame, rotated into the source frame
  const float d0 = fmaf(R[0], tx, fmaf(R[3], ty, R[6] * tz));
  const float d1 = fmaf(R[1], tx, fmaf(R[4], ty, R[7] * tz));
  const float d2 = fmaf(R[2], tx, fmaf(R[5], ty, R[8] * tz));
  // M' = R^T C' R + C_k (upper triangle)
  float m00, m01, m02, m11, m12, m22;
  fused_cov(R, r1, r2, c, m00, m01, m02, m11, m12, m22);
  // W' = adj(M') / det(M')
  const float i00 = fmaf(m11, m22, -m12 * m12);
  const float i01 = fmaf(m02, m12, -m01 * m22);
  const float i02 = fmaf(m01, m12, -m02 * m11);
  const float i11 = fmaf(m00, m22, -m02 * m02);
  const float i12 = fmaf(m01, m02, -m00 * m12);
  const float i22 = fmaf(m00, m11, -m01 * m01);
  const float det = fmaf(m00, i00, fmaf(m01, i01, m02 * i02));
  const float s = rcp_approx(det);
  const float w00 = i00 * s, w01 = i01 * s, w02 = i02 * s;
  const float w11 = i11 * s, w12 = i12 * s, w22 = i22 * s;
  // u = W' d'
  const float u0 = fmaf(w00, d0, fmaf(w01, d1, w02 * d2));
  const float u1 = fmaf(w01, d0, fmaf(w11, d1, w12 * d2));
  const float u2 = fmaf(w02, d0, fmaf(w12, d1, w22 * d2));
  // err
  acc[27] = fmaf(d0, u0, fmaf(d1, u1, fmaf(d2, u2, acc[27])));
  // b = [u x mu ; -u]
  acc[21] = fmaf(u1, z, fmaf(-u2, y, acc[21]));
  acc[22] = fmaf(u2, x, fmaf(-u0, z, acc[22]));
  acc[23] = fmaf(u0, y, fmaf(-u1, x, acc[23]));
  acc[24] -= u0;
  acc[25] -= u1;
  acc[26] -= u2;
  // H_vv = W'
  acc[15] += w00; acc[16] += w01; acc[17] += w02;
  acc[18] += w11; acc[19] += w12; acc[20] += w22;
  // P = [mu]x W'  (rows: (-z W1 + y W2), (z W0 - x W2), (-y W0 + x W1))
  const float p00 = fmaf(y, w02, -z * w01), p01 = fmaf(y, w12, -z * w11), p02 = fmaf(y, w22, -z * w12);
  const float p10 = fmaf(z, w00, -x * w02), p11 = fmaf(z, w01, -x * w12), p12 = fmaf(z, w02, -x * w22);
  const float p20 = fmaf(x, w01, -y * w00), p21 = fmaf(x, w11, -y * w01), p22 = fmaf(x, w12, -y * w02);
  acc[6] += p00; acc[7] += p01; acc[8] += p02;
  acc[9] += p10; acc[10] += p11; acc[11] += p12;
  acc[12] += p20; acc[13] += p21; acc[14] += p22;
  // H_ww = -P [mu]x
  acc[0] = fmaf(p02, y, fmaf(-p01, z, acc[0]));
  acc[1] = fmaf(p00, z, fmaf(-p02, x, acc[1]));
  acc[2] = fmaf(p01, x, fmaf(-p00, y, acc[2]));
  acc[3] = fmaf(p10, z, fmaf(-p12, x, acc[3]));
  acc[4] = fmaf(p11, x, fmaf(-p10, y, acc[4]));
  acc[5] = fmaf(p21, x, fmaf(-p20, y, acc[5]));
}

__device__ __forceinline__ void add_term(float* acc, const Pose32& P, float x, float y, float z,
                                         const float* c, float qx, float qy, float qz,
                                         const float4 r0, const float4 r1, const float4 r2) {
  add_term_t(acc, P.R, x, y, z, c, r0.x - qx, r0.y - qy, r0.z - qz, r1, r2);
  acc[28] += 1.0f;
}


// Launch-shape constants (compile-time; overridable for tuning builds).
#ifndef VGICP_NCW
#define VGICP_NCW 4
#endif
#ifndef VGICP_PTS_PER_LANE
#define VGICP_PTS_PER_LANE 2
#endif
#ifndef VGICP_STAGES
#define VGICP_STAGES 4
#endif
#ifndef VGICP_MIN_BLOCKS
#define VGICP_MIN_BLOCKS 3
#endif

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and bulk asynchronous copy (global -> shared)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps until the phase completes
// (or the hint expires) instead of spinning on the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after limit_ns (2 s by default: a bug, never a normal
// state; a test launch may set a shorter limit).
constexpr uint64_t kWaitLimitNs = 2000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// L2 policies: the source stream is read once per factor (evict first), while
// the lookup tables are re-read by every source point of the factors that
// target them (evict last).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
// 4-byte asynchronous copy global -> shared, completion tracked by an mbarrier
// through cp_async_arrive_noinc.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void consumer_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(VGICP_NCW * 32) : "memory");
}

// ---------------------------------------------------------------------------
// 1-neighbour kernel with shared-memory staging
// ---------------------------------------------------------------------------
namespace tma {
constexpr int kNCW = VGICP_NCW;               // consumer warps
constexpr int kThreads = (kNCW + 1) * 32;     // + one producer warp
constexpr int kPtsPerLane = VGICP_PTS_PER_LANE;
constexpr int kWarpPts = 32 * kPtsPerLane;    // 64 points per consumer warp
constexpr int kTile = kNCW * kWarpPts;        // 256 points per tile
constexpr int kStages = VGICP_STAGES;
constexpr int kXyzBytes = kTile * 12 + 32;    // + room for a 16-B alignment shift
constexpr int kCovBytes = kTile * 24 + 32;
constexpr int kFirst = 1, kLast = 2;

struct TileDesc {
  int32_t pair, begin, n, item, flags, xyz_off, cov_off, pad;
};

struct __align__(16) Smem {
  float4 hits[kNCW][kWarpPts * 3];            // staged voxel records of hits
  unsigned char xyz[kStages][kXyzBytes];
  unsigned char cov[kStages][kCovBytes];
  TileDesc desc[kStages];
  uint64_t full[kStages];
  uint64_t empty[kStages];
  float red[kNCW][32];
};
static_assert(kXyzBytes % 16 == 0 && kCovBytes % 16 == 0, "bulk-copy alignment");

// Copy the float range [gs, ge) of global memory into shared memory at
// dst + (gs - floor16(gs)): the 16-B aligned interior with one bulk copy
// (issue_bulk), the ragged head and tail (< 16 B each) with 4-byte cp.async
// (!issue_bulk).  Returns the bulk bytes.
__device__ __forceinline__ uint32_t stage_range(unsigned char* dst, uintptr_t gs, uintptr_t ge,
                                                uint64_t* bar, bool issue_bulk, uint64_t policy) {
  const uintptr_t g0 = gs & ~(uintptr_t)15;
  const uintptr_t a = (gs + 15) & ~(uintptr_t)15;
  const uintptr_t b = ge & ~(uintptr_t)15;
  uint32_t bulk = 0;
  uintptr_t h1 = ge, t0 = ge;
  if (b > a) {
    bulk = (uint32_t)(b - a);
    h1 = a;
    t0 = b;
    if (issue_bulk) bulk_g2s(dst + (a - g0), reinterpret_cast<const void*>(a), bulk, bar, policy);
  }
  if (!issue_bulk) {
    for (uintptr_t p = gs; p < h1; p += 4)
      cp_async4(dst + (p - g0), reinterpret_cast<const void*>(p));
    for (uintptr_t p = t0; p < ge; p += 4)
      cp_async4(dst + (p - g0), reinterpret_cast<const void*>(p));
  }
  return bulk;
}

__device__ __forceinline__ void item_bounds(const LinLaunch& L, int it, int& pair, int& b,
                                            int& e) {
  if (L.items) {
    const WorkItem w = L.items[it];
    pair = w.pair;
    b = w.begin;
    e = w.end;
  } else {
    pair = 0;
    b = it * L.item_size;
    e = (int)min((int64_t)b + L.item_size, L.single_src.n);
  }
}

// Warp reduce-scatter of 32 values: afterwards lane l holds the warp total of v[l]
// (31 shuffles instead of 5 per value).
template <int W>
__device__ __forceinline__ void rs_step(float* v, int lane) {
  const bool up = (lane & W) != 0;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    const float send = up ? v[j] : v[j + W];
    const float keep = up ? v[j + W] : v[j];
    v[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, W);
  }
}

__global__ void __launch_bounds__(kThreads, VGICP_MIN_BLOCKS) linearize_tma_kernel(const __grid_constant__ LinLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&S.full[s], 2);  // producer arrive + cp.async completion arrive
      mbar_init(&S.empty[s], kNCW);
    }
    mbar_fence_init();
  }
  __syncthreads();

  const uint64_t wait_ns = L.wait_limit_ns > 0 ? (uint64_t)L.wait_limit_ns : kWaitLimitNs;
  if (warp == kNCW) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    const uint64_t stream_pol = policy_evict_first();
    uint32_t u = 0;  // tiles issued
    bool ok = true, withheld = false;
    for (int it = blockIdx.x; it < L.n_items && ok && !withheld; it += gridDim.x) {
      int pair, b, e;
      item_bounds(L, it, pair, b, e);
      const PairDesc* pd = L.pairs ? L.pairs + pair : &L.single;
      const SrcDesc sd = L.srcs ? L.srcs[pd->src] : L.single_src;
      for (int t0 = b; t0 < e; t0 += kTile) {
        const int s = u % kStages;
        if (u >= kStages && !mbar_wait(&S.empty[s], ((u / kStages) - 1) & 1, wait_ns)) {
          ok = false;
          break;
        }
        if (L.test_withhold_tile > 0 && u + 1 == (uint32_t)L.test_withhold_tile) {
          // test launch: this tile is never issued (no copy, no arrival), so the
          // consumers' bounded wait for it runs out
          withheld = true;
          break;
        }
        const int n = min(kTile, e - t0);
        const uintptr_t xs = reinterpret_cast<uintptr_t>(sd.pts + 3 * (int64_t)t0);
        const uintptr_t cs = reinterpret_cast<uintptr_t>(sd.covs + 6 * (int64_t)t0);
        // head/tail cp.async and the descriptor, then the two arrivals, then bulk
        const uintptr_t xe = xs + 12 * (uintptr_t)n, ce = cs + 24 * (uintptr_t)n;
        const uint32_t tx = stage_range(S.xyz[s], xs, xe, &S.full[s], false, stream_pol) +
                            stage_range(S.cov[s], cs, ce, &S.full[s], false, stream_pol);
        TileDesc d;
        d.pair = pair;
        d.begin = t0;
        d.n = n;
        d.item = it;
        d.flags = (t0 == b ? kFirst : 0) | (t0 + kTile >= e ? kLast : 0);
        d.xyz_off = (int)(xs & 15);
        d.cov_off = (int)(cs & 15);
        d.pad = 0;
        S.desc[s] = d;
        cp_async_arrive_noinc(&S.full[s]);
        mbar_arrive_expect_tx(&S.full[s], tx);
        stage_range(S.xyz[s], xs, xe, &S.full[s], true, stream_pol);
        stage_range(S.cov[s], cs, ce, &S.full[s], true, stream_pol);
        ++u;
      }
    }
    if (ok && !withheld) {
      const int s = u % kStages;
      if (u >= kStages && !mbar_wait(&S.empty[s], ((u / kStages) - 1) & 1, wait_ns)) ok = false;
      if (ok) {
        S.desc[s].n = -1;
        mbar_arrive(&S.full[s]);
        mbar_arrive(&S.full[s]);
        ++u;
      }
    }
    if (!ok) atomicExch(L.status, 1);
    if (!ok || withheld) {
      // let copies already in flight land before the block exits
      for (uint32_t v = (u > kStages ? u - kStages : 0); v < u; ++v)
        mbar_wait(&S.full[v % kStages], (v / kStages) & 1, wait_ns);
    }
    return;
  }

  // ---------------- consumers ----------------
  float acc[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.0f;
  Pose32 P;
  MapDesc md;
  const PairDesc* pd = nullptr;
  uint32_t vbase = 0, mask = 0;
  float4* H = S.hits[warp];
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t map_pol = policy_evict_last();

  for (uint32_t u = 0;; ++u) {
    const int s = u % kStages;
    if (!mbar_wait(&S.full[s], (u / kStages) & 1, wait_ns)) {
      atomicExch(L.status, 1);
      break;
    }
    const TileDesc d = S.desc[s];
    if (d.n < 0) break;
    if (d.flags & kFirst) {
      pd = L.pairs ? L.pairs + d.pair : &L.single;
#pragma unroll
      for (int k = 0; k < 9; ++k) P.R[k] = pd->R[k];
      P.t[0] = pd->t[0];
      P.t[1] = pd->t[1];
      P.t[2] = pd->t[2];
      P.tmax = pd->tmax;
      md = L.maps ? L.maps[pd->map] : L.single_map;
      mask = *md.vmask;
      if (L.corr_out) vbase = *md.vbase;
    }
    const float* X = reinterpret_cast<const float*>(S.xyz[s] + d.xyz_off);
    const float* C = reinterpret_cast<const float*>(S.cov[s] + d.cov_off);

    // ---- lookup: key, first probe (two 256-bit loads) of every point, resolve ----
    int idx[kPtsPerLane];
    int kx[kPtsPerLane], ky[kPtsPerLane], kz[kPtsPerLane];
    bool live[kPtsPerLane];
    unsigned long long key[kPtsPerLane];
    uint32_t h[kPtsPerLane];
    uint32_t sa[kPtsPerLane][8], sb[kPtsPerLane][8];
#pragma unroll
    for (int k = 0; k < kPtsPerLane; ++k) {
      idx[k] = warp * kWarpPts + k * 32 + lane;
      live[k] = idx[k] < d.n;
      kx[k] = ky[k] = kz[k] = kKeyMin - 1;
      if (live[k]) {
        const float x = X[3 * idx[k]], y = X[3 * idx[k] + 1], z = X[3 * idx[k] + 2];
        const float qx = fmaf(P.R[0], x, fmaf(P.R[1], y, fmaf(P.R[2], z, P.t[0])));
        const float qy = fmaf(P.R[3], x, fmaf(P.R[4], y, fmaf(P.R[5], z, P.t[1])));
        const float qz = fmaf(P.R[6], x, fmaf(P.R[7], y, fmaf(P.R[8], z, P.t[2])));
        source_key(P, pd, md, x, y, z, qx, qy, qz, kx[k], ky[k], kz[k]);
        live[k] = key_in_range(kx[k]) && key_in_range(ky[k]) && key_in_range(kz[k]);
      }
      key[k] = live[k] ? pack_key(kx[k], ky[k], kz[k]) : kEmptyKey;
      h[k] = hash_key(kx[k], ky[k], kz[k]) & mask;
      if (live[k]) {
        ld_v8(md.vslots + h[k], map_pol, sa[k]);
        ld_v8(reinterpret_cast<const char*>(md.vslots + h[k]) + 32, map_pol, sb[k]);
      } else {
        sa[k][0] = sa[k][1] = 0xFFFFFFFFu;
      }
    }
    int vid[kPtsPerLane];
    float4 r0[kPtsPerLane], r1[kPtsPerLane], r2[kPtsPerLane];
#pragma unroll
    for (int k = 0; k < kPtsPerLane; ++k) {
      vid[k] = -1;
      if (live[k]) {
        unsigned long long t = slot_key(sa[k]);
        uint32_t hh = h[k];
        for (int p = 1; t != key[k] && t != kEmptyKey && (p > 1 || sa[k][kSlotSpill] != 0u) &&
                        p < md.max_probe;
             ++p) {
          hh = (hh + 1) & mask;
          ld_v8(md.vslots + hh, map_pol, sa[k]);
          ld_v8(reinterpret_cast<const char*>(md.vslots + hh) + 32, map_pol, sb[k]);
          t = slot_key(sa[k]);
        }
        if (t == key[k]) {
          vid[k] = (int)sa[k][kSlotVid];
          r0[k] = make_float4(__uint_as_float(sa[k][kSlotMu]), __uint_as_float(sa[k][kSlotMu + 1]),
                              __uint_as_float(sa[k][kSlotMu + 2]), 0.f);
          r1[k] = make_float4(__uint_as_float(sb[k][0]), __uint_as_float(sb[k][1]),
                              __uint_as_float(sb[k][2]), __uint_as_float(sb[k][3]));
          r2[k] = make_float4(__uint_as_float(sb[k][4]), __uint_as_float(sb[k][5]), 0.f, 0.f);
        }
      }
      if (idx[k] < d.n && (L.corr_out || L.qkey_out)) {
        const int64_t p = (int64_t)d.begin + idx[k];
        if (L.corr_out) L.corr_out[p] = vid[k] < 0 ? -1 : (int)((uint32_t)vid[k] - vbase);
        if (L.qkey_out) {
          L.qkey_out[3 * p + 0] = kx[k];
          L.qkey_out[3 * p + 1] = ky[k];
          L.qkey_out[3 * p + 2] = kz[k];
        }
      }
    }
    // ---- stage the records of the hits, compacted per warp ----
    int nh = 0;
#pragma unroll
    for (int k = 0; k < kPtsPerLane; ++k) {
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, vid[k] >= 0);
      if (vid[k] >= 0) {
        const int pos = nh + __popc(m & lt_mask);
        H[3 * pos + 0] = make_float4(r0[k].x, r0[k].y, r0[k].z, __int_as_float(idx[k]));
        H[3 * pos + 1] = r1[k];
        H[3 * pos + 2] = r2[k];
      }
      nh += __popc(m);
    }
    __syncwarp();
    // ---- terms of the hits, from shared memory ----
    for (int j = lane; j < nh; j += 32) {
      const float4 e0 = H[3 * j], e1 = H[3 * j + 1], e2 = H[3 * j + 2];
      const int i = __float_as_int(e0.w);
      const float x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
      const float2* cv = reinterpret_cast<const float2*>(C + 6 * i);
      const float2 c01 = cv[0], c23 = cv[1], c45 = cv[2];
      const float c[6] = {c01.x, c01.y, c23.x, c23.y, c45.x, c45.y};
      const float qx = fmaf(P.R[0], x, fmaf(P.R[1], y, fmaf(P.R[2], z, P.t[0])));
      const float qy = fmaf(P.R[3], x, fmaf(P.R[4], y, fmaf(P.R[5], z, P.t[1])));
      const float qz = fmaf(P.R[6], x, fmaf(P.R[7], y, fmaf(P.R[8], z, P.t[2])));
      add_term(acc, P, x, y, z, c, qx, qy, qz, e0, e1, e2);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.empty[s]);

    if (d.flags & kLast) {
      rs_step<16>(acc, lane);
      rs_step<8>(acc, lane);
      rs_step<4>(acc, lane);
      rs_step<2>(acc, lane);
      rs_step<1>(acc, lane);
      S.red[warp][lane] = acc[0];
      consumer_bar();
      if (warp == 0 && lane < kAcc) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kNCW; ++w) t += (double)S.red[w][lane];
        L.partials[(int64_t)d.item * kPartialStride + lane] = t;
      }
      consumer_bar();
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[k] = 0.0f;
    }
  }
}

}  // namespace tma

// ---------------------------------------------------------------------------
// One point per thread (1 or 27 neighbours); the lookups and records come from
// global memory through L1.
// ---------------------------------------------------------------------------
// Cost and gradient of one term, for the differentiable interface:
//   MODE 1: err only;  MODE 2: + g = 2 J^T W d (W held, the Gauss-Newton gradient);
//   MODE 3: + the change of W with the rotation: for omega_i the exact derivative
//           adds -u^T dM/domega_i u = 2 (u' x C_k u')_i, u' = W' d' (source frame).
// Accumulators: 0..5 gradient, 6 err, 28 inlier count.
template <int MODE>
__device__ __forceinline__ void eval_term(float* acc, const Pose32& P, float x, float y, float z,
                                          const float* c, float qx, float qy, float qz,
                                          const float4 r0, const float4 r1, const float4 r2) {
  const float* R = P.R;
  const float tx = r0.x - qx, ty = r0.y - qy, tz = r0.z - qz;
  const float d0 = fmaf(R[0], tx, fmaf(R[3], ty, R[6] * tz));
  const float d1 = fmaf(R[1], tx, fmaf(R[4], ty, R[7] * tz));
  const float d2 = fmaf(R[2], tx, fmaf(R[5], ty, R[8] * tz));
  float m00, m01, m02, m11, m12, m22;
  fused_cov(R, r1, r2, c, m00, m01, m02, m11, m12, m22);
  const float i00 = fmaf(m11, m22, -m12 * m12);
  const float i01 = fmaf(m02, m12, -m01 * m22);
  const float i02 = fmaf(m01, m12, -m02 * m11);
  const float i11 = fmaf(m00, m22, -m02 * m02);
  const float i12 = fmaf(m01, m02, -m00 * m12);
  const float i22 = fmaf(m00, m11, -m01 * m01);
  const float det = fmaf(m00, i00, fmaf(m01, i01, m02 * i02));
  const float sc = rcp_approx(det);
  const float u0 = fmaf(i00, d0, fmaf(i01, d1, i02 * d2)) * sc;
  const float u1 = fmaf(i01, d0, fmaf(i11, d1, i12 * d2)) * sc;
  const float u2 = fmaf(i02, d0, fmaf(i12, d1, i22 * d2)) * sc;
  acc[6] = fmaf(d0, u0, fmaf(d1, u1, fmaf(d2, u2, acc[6])));
  if (MODE >= 2) {
    acc[0] = fmaf(2.0f * u1, z, fmaf(-2.0f * u2, y, acc[0]));
    acc[1] = fmaf(2.0f * u2, x, fmaf(-2.0f * u0, z, acc[1]));
    acc[2] = fmaf(2.0f * u0, y, fmaf(-2.0f * u1, x, acc[2]));
    acc[3] -= 2.0f * u0;
    acc[4] -= 2.0f * u1;
    acc[5] -= 2.0f * u2;
  }
  if (MODE == 3) {
    const float k0 = fmaf(c[0], u0, fmaf(c[1], u1, c[2] * u2));
    const float k1 = fmaf(c[1], u0, fmaf(c[3], u1, c[4] * u2));
    const float k2 = fmaf(c[2], u0, fmaf(c[4], u1, c[5] * u2));
    acc[0] = fmaf(2.0f * u1, k2, fmaf(-2.0f * u2, k1, acc[0]));
    acc[1] = fmaf(2.0f * u2, k0, fmaf(-2.0f * u0, k2, acc[1]));
    acc[2] = fmaf(2.0f * u0, k1, fmaf(-2.0f * u1, k0, acc[2]));
  }
  acc[28] += 1.0f;
}

// MODE 0: linearization (H, b, err); 1-3: cost / gradient / exact gradient;
// 4: overlap (the inlier count only: no term arithmetic, no covariance reads).
template <int MODE>
__device__ __forceinline__ void term(float* acc, const Pose32& P, float x, float y, float z,
                                     const float* c, float qx, float qy, float qz,
                                     const float4 r0, const float4 r1, const float4 r2) {
  if (MODE == 0)
    add_term(acc, P, x, y, z, c, qx, qy, qz, r0, r1, r2);
  else if (MODE == 4)
    acc[28] += 1.0f;
  else
    eval_term<MODE>(acc, P, x, y, z, c, qx, qy, qz, r0, r1, r2);
}

// ---------------------------------------------------------------------------
// Per-point kernel: one source point per thread, dynamically scheduled work
// items.  Occupancy is what hides the DRAM latency of the stream and the L2
// latency of the lookup here, so the kernel keeps its registers for the 28
// accumulators and the term arithmetic: the constants of the current work item
// (pose, map and source descriptors) sit in shared memory and are re-read
// (volatile) in every iteration instead of living in registers across the
// point loop.
// ---------------------------------------------------------------------------
#ifndef VGICP_SIMPLE_MIN_BLOCKS
#define VGICP_SIMPLE_MIN_BLOCKS 3
#endif

struct __align__(16) ItemConst {
  float R[9];
  float t[3];                 // R, t: 3 float4
  float tmax, inv_r, margin_scale;
  uint32_t mask;              // float4 #3
  const VSlot* vslots;
  const float* pts;           // #4
  const float* covs;
  const PairDesc* pd;         // #5
  double r;
  int32_t max_probe, pad;     // #6
};

__device__ __forceinline__ float4 lds_f4(const void* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ void lds_2ptr(const void* p, uint64_t& a, uint64_t& b) {
  asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];"
               : "=l"(a), "=l"(b)
               : "r"((uint32_t)__cvta_generic_to_shared(p)));
}

template <int NEIGH, int MODE, bool DBG>
__global__ void __launch_bounds__(kSimpleThreads, VGICP_SIMPLE_MIN_BLOCKS)
    linearize_simple_kernel(const __grid_constant__ LinLaunch L) {
  __shared__ float red[kSimpleThreads / 32][kAcc];
  // 27 neighbours: each thread's hits (slot offsets) of its current point
  __shared__ uint32_t hits[NEIGH == 27 ? 27 * kSimpleThreads : 1];
  __shared__ ItemConst ic;
  __shared__ int next_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t pol = policy_evict_last_l();

  for (int it = blockIdx.x; it < L.n_items;) {
    int pair, begin, end;
    tma::item_bounds(L, it, pair, begin, end);
    if (threadIdx.x == 0) {
      const PairDesc* pd = L.pairs ? L.pairs + pair : &L.single;
      const MapDesc md = L.maps ? L.maps[pd->map] : L.single_map;
      const SrcDesc sd = L.srcs ? L.srcs[pd->src] : L.single_src;
#pragma unroll
      for (int k = 0; k < 9; ++k) ic.R[k] = pd->R[k];
      ic.t[0] = pd->t[0];
      ic.t[1] = pd->t[1];
      ic.t[2] = pd->t[2];
      ic.tmax = pd->tmax;
      ic.inv_r = md.inv_r;
      ic.margin_scale = md.margin_scale;
      ic.mask = *md.vmask;
      ic.vslots = md.vslots;
      ic.pts = sd.pts;
      ic.covs = sd.covs;
      ic.pd = pd;
      ic.r = md.r;
      ic.max_probe = md.max_probe;
    }
    uint32_t vbase = 0;
    if (DBG && L.corr_out) {
      const PairDesc* pd = L.pairs ? L.pairs + pair : &L.single;
      vbase = *(L.maps ? L.maps[pd->map] : L.single_map).vbase;
    }
    __syncthreads();

    float acc[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k] = 0.0f;

    for (int p = begin + threadIdx.x; p < end; p += kSimpleThreads) {
      const float4 g0 = lds_f4(&ic.R[0]), g1 = lds_f4(&ic.R[4]), g2 = lds_f4(&ic.R[8]);
      const float4 g3 = lds_f4(&ic.tmax);
      uint64_t vs, ps, cs, pds;
      lds_2ptr(&ic.vslots, vs, ps);
      lds_2ptr(&ic.covs, cs, pds);
      Pose32 P;
      P.R[0] = g0.x; P.R[1] = g0.y; P.R[2] = g0.z; P.R[3] = g0.w;
      P.R[4] = g1.x; P.R[5] = g1.y; P.R[6] = g1.z; P.R[7] = g1.w;
      P.R[8] = g2.x;
      P.t[0] = g2.y; P.t[1] = g2.z; P.t[2] = g2.w;
      P.tmax = g3.x;
      MapDesc md;
      md.vslots = reinterpret_cast<const VSlot*>(vs);
      md.inv_r = g3.y;
      md.margin_scale = g3.z;
      const uint32_t mask = __float_as_uint(g3.w);
      const PairDesc* pd = reinterpret_cast<const PairDesc*>(pds);

      const float* pt = reinterpret_cast<const float*>(ps) + 3 * (int64_t)p;
      const float x = __ldg(pt + 0), y = __ldg(pt + 1), z = __ldg(pt + 2);
      const float2* cv = reinterpret_cast<const float2*>(reinterpret_cast<const float*>(cs) +
                                                         6 * (int64_t)p);
      const float2 c01 = __ldg(cv + 0), c23 = __ldg(cv + 1), c45 = __ldg(cv + 2);
      const float c[6] = {c01.x, c01.y, c23.x, c23.y, c45.x, c45.y};
      const float qx = fmaf(P.R[0], x, fmaf(P.R[1], y, fmaf(P.R[2], z, P.t[0])));
      const float qy = fmaf(P.R[3], x, fmaf(P.R[4], y, fmaf(P.R[5], z, P.t[1])));
      const float qz = fmaf(P.R[6], x, fmaf(P.R[7], y, fmaf(P.R[8], z, P.t[2])));
      int kx, ky, kz;
      {
        // the binary64 fallback reads r from shared memory only when taken
        const float S = fabsf(x) + fabsf(y) + fabsf(z) + P.tmax;
        const float m = fmaf(S, md.margin_scale, 1.1920928955078125e-7f);
        const float yx = qx * md.inv_r, yy = qy * md.inv_r, yz = qz * md.inv_r;
        const float fx = floorf(yx), fy = floorf(yy), fz = floorf(yz);
        const float rx = yx - fx, ry = yy - fy, rz = yz - fz;
        const bool ax = (rx < m) | (rx > 1.0f - m);
        const bool ay = (ry < m) | (ry > 1.0f - m);
        const bool az = (rz < m) | (rz > 1.0f - m);
        kx = clamp_to_int(fx);
        ky = clamp_to_int(fy);
        kz = clamp_to_int(fz);
        if (ax | ay | az) {
          MapDesc mr;
          mr.r = ic.r;
          if (ax) kx = axis_key_f64(pd, mr, 0, x, y, z);
          if (ay) ky = axis_key_f64(pd, mr, 1, x, y, z);
          if (az) kz = axis_key_f64(pd, mr, 2, x, y, z);
        }
      }
      if (DBG && L.qkey_out) {
        L.qkey_out[3 * (int64_t)p + 0] = kx;
        L.qkey_out[3 * (int64_t)p + 1] = ky;
        L.qkey_out[3 * (int64_t)p + 2] = kz;
      }
      md.max_probe = ic.max_probe;
      if (NEIGH == 1) {
        float4 a0, a1, a2;
        const int vid = lookup(md, mask, kx, ky, kz, pol, a0, a1, a2);
        if (DBG && L.corr_out) L.corr_out[p] = vid < 0 ? -1 : (int)((uint32_t)vid - vbase);
        if (vid >= 0) term<MODE>(acc, P, x, y, z, c, qx, qy, qz, a0, a1, a2);
        continue;
      }
      if (DBG && L.corr_out) {
        float4 a0, a1, a2;
        const int own = lookup(md, mask, kx, ky, kz, pol, a0, a1, a2);
        L.corr_out[p] = own < 0 ? -1 : (int)((uint32_t)own - vbase);
      }
      // the 27 probes first, hits recorded; then the terms, hit by hit, so a
      // warp evaluates a term while most of its lanes still have one.  The
      // probes go a row of three neighbours at a time, their home slots' first
      // 16 B (key, spill flag) loaded together; a miss whose home slot holds
      // another key with its spill flag set probes on
      int nh = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy) {
          const int yy = ky + dy, zz = kz + dz;
          const bool row_ok = key_in_range(yy) && key_in_range(zz);
          uint32_t A[3][4];
          uint32_t hh[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            hh[j] = hash_key(kx + j - 1, yy, zz) & mask;
            ld_v4(md.vslots + hh[j], pol, A[j]);
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const int xx = kx + j - 1;
            if (!row_ok || !key_in_range(xx)) continue;
            const unsigned long long key = pack_key(xx, yy, zz);
            const unsigned long long k0 =
                (unsigned long long)A[j][0] | ((unsigned long long)A[j][1] << 32);
            int hs = -1;
            if (k0 == key) {
              hs = (int)hh[j];
            } else if (k0 != kEmptyKey && A[j][kSlotSpill] != 0u) {
              uint32_t h = (hh[j] + 1) & mask;  // spilled keys: probe on
              for (int q = 1; q < md.max_probe; ++q) {
                uint32_t a[4];
                ld_v4(md.vslots + h, pol, a);
                const unsigned long long k =
                    (unsigned long long)a[0] | ((unsigned long long)a[1] << 32);
                if (k == key) { hs = (int)h; break; }
                if (k == kEmptyKey) break;
                h = (h + 1) & mask;
              }
            }
            if (hs >= 0) hits[27 * threadIdx.x + nh++] = (uint32_t)hs;
          }
        }
      for (int k = 0; k < nh; ++k) {
        const VSlot* t = md.vslots + hits[27 * threadIdx.x + k];
        // count and mu' (bytes 16..31), then L (bytes 32..63)
        uint32_t a[4], b[8];
        ld_v4(reinterpret_cast<const char*>(t) + 16, pol, a);
        ld_v8(reinterpret_cast<const char*>(t) + 32, pol, b);
        const float4 a0 = make_float4(__uint_as_float(a[1]), __uint_as_float(a[2]),
                                      __uint_as_float(a[3]), 0.f);
        const float4 a1 = make_float4(__uint_as_float(b[0]), __uint_as_float(b[1]),
                                      __uint_as_float(b[2]), __uint_as_float(b[3]));
        const float4 a2 = make_float4(__uint_as_float(b[4]), __uint_as_float(b[5]), 0.f, 0.f);
        term<MODE>(acc, P, x, y, z, c, qx, qy, qz, a0, a1, a2);
      }
    }

#pragma unroll
    for (int k = 0; k < kAcc; ++k) {
      float v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      acc[k] = v;
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < kAcc; ++k) red[warp][k] = acc[k];
    }
    if (threadIdx.x == 0) next_item = (int)gridDim.x + atomicAdd(L.status + 1, 1);
    __syncthreads();
    if (threadIdx.x < kAcc) {
      double s = 0.0;
      for (int w = 0; w < kSimpleThreads / 32; ++w) s += (double)red[w][threadIdx.x];
      L.partials[(int64_t)it * kPartialStride + threadIdx.x] = s;
    }
    it = next_item;  // read between the two barriers; rewritten only after the second
    __syncthreads();
  }
}

template <int NEIGH, int MODE>
void launch_simple(const LinLaunch& L, int grid, cudaStream_t st) {
  if (L.corr_out || L.qkey_out)
    linearize_simple_kernel<NEIGH, MODE, true><<<grid, kSimpleThreads, 0, st>>>(L);
  else
    linearize_simple_kernel<NEIGH, MODE, false><<<grid, kSimpleThreads, 0, st>>>(L);
}

// ---------------------------------------------------------------------------
// Hit-compacting per-warp kernel (1 neighbour).  The lookup phase runs one
// point per lane; the lanes whose voxel exists push (point, covariance, target-
// frame residual mu' - q, voxel covariance) as one 80-B entry into their warp's
// queue in shared memory.  Whenever 32 entries are queued the warp evaluates
// them with every lane busy, so lanes whose point missed do not cost term
// arithmetic.  Item constants live in shared memory as in the per-point kernel.
// ---------------------------------------------------------------------------
namespace compact {
#ifndef VGICP_COMPACT_MIN_BLOCKS
#define VGICP_COMPACT_MIN_BLOCKS 3
#endif
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kQueue = 64;  // entries per warp (< 32 left after a drain + at most 32 pushed)

__device__ __forceinline__ void eval_entry(float* acc, const float* R, const float4* E) {
  const float4 e0 = E[0], e1 = E[1], e2 = E[2], e3 = E[3], e4 = E[4];
  const float c[6] = {e0.w, e1.x, e1.y, e1.z, e1.w, e2.x};
  add_term_t(acc, R, e0.x, e0.y, e0.z, c, e2.y, e2.z, e2.w, e3, e4);
}

__global__ void __launch_bounds__(kThreads, VGICP_COMPACT_MIN_BLOCKS)
    linearize_compact_kernel(const __grid_constant__ LinLaunch L) {
  __shared__ __align__(16) float4 queue[kWarps][kQueue * 5];
  __shared__ float red[kWarps][kAcc];
  __shared__ ItemConst ic;
  __shared__ int next_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t pol = policy_evict_last_l();
  float4* Q = queue[warp];

  for (int it = blockIdx.x; it < L.n_items;) {
    int pair, begin, end;
    tma::item_bounds(L, it, pair, begin, end);
    if (threadIdx.x == 0) {
      const PairDesc* pd = L.pairs ? L.pairs + pair : &L.single;
      const MapDesc md = L.maps ? L.maps[pd->map] : L.single_map;
      const SrcDesc sd = L.srcs ? L.srcs[pd->src] : L.single_src;
#pragma unroll
      for (int k = 0; k < 9; ++k) ic.R[k] = pd->R[k];
      ic.t[0] = pd->t[0];
      ic.t[1] = pd->t[1];
      ic.t[2] = pd->t[2];
      ic.tmax = pd->tmax;
      ic.inv_r = md.inv_r;
      ic.margin_scale = md.margin_scale;
      ic.mask = *md.vmask;
      ic.vslots = md.vslots;
      ic.pts = sd.pts;
      ic.covs = sd.covs;
      ic.pd = pd;
      ic.r = md.r;
      ic.max_probe = md.max_probe;
    }
    __syncthreads();

    float acc[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k] = 0.0f;
    int qn = 0;  // queued entries (warp-uniform)
    const int n = end - begin;

    for (int base = warp * 32; base < n; base += kThreads) {
      const int p = begin + base + lane;
      bool hit = false;
      float x = 0.f, y = 0.f, z = 0.f, tx = 0.f, ty = 0.f, tz = 0.f;
      float2 c01, c23, c45;
      float4 a1, a2;
      if (p < end) {
        const float4 g0 = lds_f4(&ic.R[0]), g1 = lds_f4(&ic.R[4]), g2 = lds_f4(&ic.R[8]);
        const float4 g3 = lds_f4(&ic.tmax);
        uint64_t vs, ps, cs, pds;
        lds_2ptr(&ic.vslots, vs, ps);
        lds_2ptr(&ic.covs, cs, pds);
        const float* pt = reinterpret_cast<const float*>(ps) + 3 * (int64_t)p;
        x = __ldg(pt + 0);
        y = __ldg(pt + 1);
        z = __ldg(pt + 2);
        const float2* cv = reinterpret_cast<const float2*>(reinterpret_cast<const float*>(cs) +
                                                           6 * (int64_t)p);
        c01 = __ldg(cv + 0);
        c23 = __ldg(cv + 1);
        c45 = __ldg(cv + 2);
        const float qx = fmaf(g0.x, x, fmaf(g0.y, y, fmaf(g0.z, z, g2.y)));
        const float qy = fmaf(g0.w, x, fmaf(g1.x, y, fmaf(g1.y, z, g2.z)));
        const float qz = fmaf(g1.z, x, fmaf(g1.w, y, fmaf(g2.x, z, g2.w)));
        const float S = fabsf(x) + fabsf(y) + fabsf(z) + g3.x;
        const float m = fmaf(S, g3.z, 1.1920928955078125e-7f);
        const float yx = qx * g3.y, yy = qy * g3.y, yz = qz * g3.y;
        const float fx = floorf(yx), fy = floorf(yy), fz = floorf(yz);
        const float rx = yx - fx, ry = yy - fy, rz = yz - fz;
        const bool ax = (rx < m) | (rx > 1.0f - m);
        const bool ay = (ry < m) | (ry > 1.0f - m);
        const bool az = (rz < m) | (rz > 1.0f - m);
        int kx = clamp_to_int(fx), ky = clamp_to_int(fy), kz = clamp_to_int(fz);
        if (ax | ay | az) {
          const PairDesc* pd = reinterpret_cast<const PairDesc*>(pds);
          MapDesc mr;
          mr.r = ic.r;
          if (ax) kx = axis_key_f64(pd, mr, 0, x, y, z);
          if (ay) ky = axis_key_f64(pd, mr, 1, x, y, z);
          if (az) kz = axis_key_f64(pd, mr, 2, x, y, z);
        }
        MapDesc md;
        md.vslots = reinterpret_cast<const VSlot*>(vs);
        md.max_probe = ic.max_probe;
        float4 a0;
        const int vid = lookup(md, __float_as_uint(g3.w), kx, ky, kz, pol, a0, a1, a2);
        hit = vid >= 0;
        tx = a0.x - qx;
        ty = a0.y - qy;
        tz = a0.z - qz;
      }
      const uint32_t hm = __ballot_sync(0xFFFFFFFFu, hit);
      if (hit) {
        float4* E = Q + 5 * (qn + __popc(hm & lt_mask));
        E[0] = make_float4(x, y, z, c01.x);
        E[1] = make_float4(c01.y, c23.x, c23.y, c45.x);
        E[2] = make_float4(c45.y, tx, ty, tz);
        E[3] = a1;
        E[4] = a2;
      }
      if (lane == 0) acc[28] += (float)__popc(hm);
      qn += __popc(hm);
      __syncwarp();
      if (qn >= 32) {  // one full warp of terms: lane l takes entry qn - 32 + l
        const float4 g0 = lds_f4(&ic.R[0]), g1 = lds_f4(&ic.R[4]), g2 = lds_f4(&ic.R[8]);
        const float R[9] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, g2.x};
        eval_entry(acc, R, Q + 5 * (qn - 32 + lane));
        qn -= 32;
        __syncwarp();
      }
    }
    if (lane < qn) {  // drain the partially filled queue
      const float4 g0 = lds_f4(&ic.R[0]), g1 = lds_f4(&ic.R[4]), g2 = lds_f4(&ic.R[8]);
      const float R[9] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, g2.x};
      eval_entry(acc, R, Q + 5 * lane);
    }
    __syncwarp();

#pragma unroll
    for (int k = 0; k < kAcc; ++k) {
      float v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      acc[k] = v;
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < kAcc; ++k) red[warp][k] = acc[k];
    }
    if (threadIdx.x == 0) next_item = (int)gridDim.x + atomicAdd(L.status + 1, 1);
    __syncthreads();
    if (threadIdx.x < kAcc) {
      double t = 0.0;
      for (int w = 0; w < kWarps; ++w) t += (double)red[w][threadIdx.x];
      L.partials[(int64_t)it * kPartialStride + threadIdx.x] = t;
    }
    it = next_item;  // read between the two barriers; rewritten only after the second
    __syncthreads();
  }
}
}  // namespace compact


// One warp per pair: lane k sums term k over the pair's items in order.  For the
// gradient modes, an optional right Jacobian per pair (jr, 36 doubles, row-major)
// maps the gradient g of the right perturbation to that of the pose increment,
// J_r^T g, and an optional per-pair scale multiplies it (the incoming gradient of
// a reverse-mode pass).
__global__ void reduce_kernel(const double* __restrict__ partials, const int2* __restrict__ span,
                              int32_t n_items_single, int64_t n_pairs,
                              const int32_t* __restrict__ status, double* __restrict__ out,
                              int64_t* __restrict__ inliers, int32_t mode,
                              const double* __restrict__ jr, const double* __restrict__ gscale) {
  const int64_t pair = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= n_pairs) return;
  const int32_t a = span ? span[pair].x : 0;
  const int32_t b = span ? span[pair].y : n_items_single;
  double s = 0.0;
  if (lane < kAcc)
    for (int32_t it = a; it < b; ++it) s += partials[(int64_t)it * kPartialStride + lane];
  if (status && *status != 0) s = __longlong_as_double(0x7FF8000000000000ll);  // NaN
  if (mode == 4) {  // overlap: the inlier count only
    if (lane == 28) inliers[pair] = (status && *status != 0) ? -1 : (int64_t)llrint(s);
    return;
  }
  if (mode != 0) {  // gradient (6) and err (1)
    if (jr && mode >= 2) {
      double g[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) g[i] = __shfl_sync(0xFFFFFFFFu, s, i);
      if (lane < 6) {
        const double* J = jr + pair * 36;
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) v = fma(J[6 * i + lane], g[i], v);
        s = gscale ? v * gscale[pair] : v;
      }
    } else if (gscale && lane < 6 && mode >= 2) {
      s *= gscale[pair];
    }
    if (lane < 7) out[pair * 7 + lane] = s;
    if (lane == 28) inliers[pair] = (status && *status != 0) ? -1 : (int64_t)llrint(s);
    return;
  }
  double* o = out + pair * 43;
  constexpr int ww_r[6] = {0, 0, 0, 1, 1, 2}, ww_c[6] = {0, 1, 2, 1, 2, 2};
  if (lane < 6) {
    o[6 * ww_r[lane] + ww_c[lane]] = s;
    o[6 * ww_c[lane] + ww_r[lane]] = s;
  } else if (lane < 15) {
    const int i = (lane - 6) / 3, j = (lane - 6) % 3;
    o[6 * i + 3 + j] = s;
    o[6 * (3 + j) + i] = s;
  } else if (lane < 21) {
    const int k = lane - 15;
    o[6 * (3 + ww_r[k]) + 3 + ww_c[k]] = s;
    o[6 * (3 + ww_c[k]) + 3 + ww_r[k]] = s;
  } else if (lane < 27) {
    o[36 + (lane - 21)] = s;
  } else if (lane == 27) {
    o[42] = s;
  } else if (lane == 28) {
    inliers[pair] = (status && *status != 0) ? -1 : (int64_t)llrint(s);
  }
}

}  // namespace

// One-shot test state for the staged kernel's bounded waits
// (vgicp_test_expire_waits): the tile its producers withhold (+1; 0 = none) and
// the wait limit of that one launch.
std::mutex g_wait_test_mu;
int32_t g_wait_test_tile = 0;
int64_t g_wait_test_ns = 0;

void take_wait_test(LinLaunch& L) {
  std::lock_guard<std::mutex> lock(g_wait_test_mu);
  if (g_wait_test_tile > 0) {
    L.test_withhold_tile = g_wait_test_tile;
    L.wait_limit_ns = g_wait_test_ns;
    g_wait_test_tile = 0;
    g_wait_test_ns = 0;
  }
}

int arm_wait_test(int32_t tile, int64_t limit_ns) {
  if (tile < 0 || limit_ns <= 0 || limit_ns > 2000000000ll)
    return set_error(VGICP_ERR_INVALID_ARG, "tile must be >= 0 and the limit in (0, 2 s]");
  std::lock_guard<std::mutex> lock(g_wait_test_mu);
  g_wait_test_tile = tile + 1;
  g_wait_test_ns = limit_ns;
  return VGICP_OK;
}

int default_item_size() { return 16384; }

int default_variant() { return 1; }

int linearize_grid(int neighbours, int variant) {
  if (variant == 0) variant = default_variant();
  if (neighbours == 27 || variant == 1) return device_sm_count() * VGICP_SIMPLE_MIN_BLOCKS;
  if (variant == 3) return device_sm_count() * VGICP_COMPACT_MIN_BLOCKS;
  return device_sm_count() * VGICP_MIN_BLOCKS;
}

int launch_linearize(const LinLaunch& L, cudaStream_t st) {
  if (L.n_items <= 0) return VGICP_OK;
  const int variant = L.mode != 0 ? 1 : (L.variant ? L.variant : default_variant());
  int grid = L.grid > 0 ? L.grid : linearize_grid(L.neighbours, variant);
  grid = std::min(grid, L.n_items);
  if (L.ev_start) VGICP_CUDA_TRY(cudaEventRecord(L.ev_start, st));
  if (L.mode != 0) {
    // cost / gradient evaluations use the per-point kernel
    if (L.neighbours == 27) {
      if (L.mode == 1) launch_simple<27, 1>(L, grid, st);
      else if (L.mode == 2) launch_simple<27, 2>(L, grid, st);
      else launch_simple<27, 3>(L, grid, st);
    } else {
      if (L.mode == 1) launch_simple<1, 1>(L, grid, st);
      else if (L.mode == 2) launch_simple<1, 2>(L, grid, st);
      else if (L.mode == 3) launch_simple<1, 3>(L, grid, st);
      else launch_simple<1, 4>(L, grid, st);
    }
  } else if (L.neighbours == 27) {
    launch_simple<27, 0>(L, grid, st);
  } else if (variant == 1) {
    launch_simple<1, 0>(L, grid, st);
  } else if (variant == 3 && !L.corr_out && !L.qkey_out) {
    compact::linearize_compact_kernel<<<grid, compact::kThreads, 0, st>>>(L);
  } else if (variant == 3) {
    launch_simple<1, 0>(L, grid, st);  // the per-point kernel writes the debug outputs

  } else {
    // the dynamic shared-memory limit is a per-device function attribute: set it
    // once per device, under a lock (host threads may launch concurrently)
    static std::mutex attr_mu;
    static bool attr_set[kMaxDevices] = {false};
    int dev = 0;
    VGICP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
      return set_error(VGICP_ERR_INVALID_ARG, "device index beyond the supported range");
    {
      std::lock_guard<std::mutex> lock(attr_mu);
      if (!attr_set[dev]) {
        VGICP_CUDA_TRY(cudaFuncSetAttribute(tma::linearize_tma_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)sizeof(tma::Smem)));
        attr_set[dev] = true;
      }
    }
    LinLaunch Lt = L;
    take_wait_test(Lt);
    tma::linearize_tma_kernel<<<grid, tma::kThreads, sizeof(tma::Smem), st>>>(Lt);
  }
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  if (L.ev_stop) VGICP_CUDA_TRY(cudaEventRecord(L.ev_stop, st));
  return VGICP_OK;
}

int launch_reduce(const double* partials, const int2* span, int32_t n_items_single,
                  int64_t n_pairs, const int32_t* status, double* out, int64_t* inliers,
                  cudaStream_t st, int32_t mode, const double* jr, const double* gscale) {
  if (n_pairs <= 0) return VGICP_OK;
  const int warps = 8;
  const int64_t blocks = (n_pairs + warps - 1) / warps;
  reduce_kernel<<<(unsigned)blocks, warps * 32, 0, st>>>(partials, span, n_items_single, n_pairs,
                                                         status, out, inliers, mode, jr, gscale);
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return VGICP_OK;
}

}  // namespace vgicp
