// Device-side definitions shared by the build and linearize kernels:
// the exact voxel key, key packing, the hash, and the table/record layouts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vgicp {

// ---------------------------------------------------------------------------
// Layouts in HBM
// ---------------------------------------------------------------------------

// Hash slot (16 B, 16-B aligned): packed key, then (vid, count).
//   key   : kEmptyKey or a packed voxel key (< 2^63)
//   vid   : during the build, the smallest point index (in the batch) of the voxel;
//           after it, the global voxel index
//   count : number of points in the voxel
struct __align__(16) Slot {
  unsigned long long key;
  uint32_t vid;
  uint32_t count;
};

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kKeyBits = 21;
constexpr int kKeyBias = 1 << (kKeyBits - 1);  // key fields hold k + 2^20
constexpr int kKeyMin = -kKeyBias;             // valid k: [-2^20, 2^20)
constexpr int kKeyMax = kKeyBias - 1;
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// Voxel record: 3 x float4 = 48 B (kept for export and tests).
//   r0 = (mu'.x, mu'.y, mu'.z, bits(N)), r1 = (C'xx, C'xy, C'xz, C'yy),
//   r2 = (C'yz, C'zz, 0, 0)
constexpr int kRecordF4 = 3;

// Lookup table slot with the voxel Gaussian inline (64 B, 64-B aligned): a
// lookup is two independent 256-bit loads; a probe that needs only the key and
// the spill flag reads the first 16 B.
//   bytes  0..15: key (u64), spill (u32), vid (u32)
//   bytes 16..31: count (u32), mu' (3 x f32)
//   bytes 32..63: L, the Cholesky factor of C' (6 x f32: l00 l10 l20 l11 l21
//                 l22), pad
// Linear probing from the key's home slot h.  spill (of slot h) is nonzero iff
// some key whose home is h lies further along the probe sequence, so a lookup
// whose home slot holds another key and has spill == 0 is a miss after one
// round trip, like a key found at home; only the rest probe on.
// Each map's table has capacity next_pow2(max(16, kLookupLoad V)) (decided on the
// device after the voxels are counted) inside a region sized for the worst case
// V = n.  The low load factor (<= 1 / kLookupLoad) keeps most keys at home.
#ifndef VGICP_LOOKUP_LOAD
#define VGICP_LOOKUP_LOAD 16
#endif
constexpr uint32_t kLookupLoad = VGICP_LOOKUP_LOAD;
struct __align__(64) VSlot {
  unsigned long long key;
  uint32_t spill;
  uint32_t vid;
  uint32_t count;
  float mu[3];
  float cov[6];
  float pad1[2];
};
static_assert(sizeof(VSlot) == 64, "VSlot is 64 B");
// 32-bit words of the first half as loaded: key 0..1, then these
constexpr int kSlotSpill = 2, kSlotVid = 3, kSlotMu = 5;

// Per-map descriptor read by the linearize kernels.
struct MapDesc {
  const VSlot* vslots;    // this map's lookup table
  const uint32_t* vmask;  // device: its capacity - 1
  int32_t max_probe;
  float inv_r;            // float32(1 / r)
  float margin_scale;     // inv_r * 2^-21 (see source_key)
  int32_t pad;
  double r;
  const uint32_t* vbase;  // first global voxel index of this map (device)
};

// Per-factor descriptor: pose in both precisions, map and source index.
struct PairDesc {
  float R[9];     // float32(R), row-major
  float t[3];     // float32(t)
  float tmax;     // max |t_i| (float32, rounded up)
  int32_t map;    // index into the MapDesc array
  int32_t src;    // index into the SrcDesc array
  int32_t pad;
  double R64[9];  // binary64 R, row-major
  double t64[3];
};

struct SrcDesc {
  const float* pts;   // n x 3
  const float* covs;  // n x 6
  int64_t n;
};

// Voxels of a map are put in Morton order in chunks of this many (one CTA sorts
// one chunk in shared memory).
constexpr int kMortonChunk = 16384;

// Work item: points [begin, end) of pair `pair`.
struct __align__(16) WorkItem {
  int32_t pair;
  int32_t begin;
  int32_t end;
  int32_t pad;
};

// Number of float accumulators per factor: H (21 unique), b (6), err (1),
// plus the inlier count (carried as a float inside a block, exact below 2^24).
constexpr int kTerms = 28;
constexpr int kAcc = kTerms + 1;
constexpr int kPartialStride = 32;  // doubles per partial record

// ---------------------------------------------------------------------------
// Voxel key: k = floor(x / r) as if evaluated in binary64.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long pack_key(int kx, int ky, int kz) {
  return ((unsigned long long)(uint32_t)(kx + kKeyBias) << (2 * kKeyBits)) |
         ((unsigned long long)(uint32_t)(ky + kKeyBias) << kKeyBits) |
         (unsigned long long)(uint32_t)(kz + kKeyBias);
}

__device__ __forceinline__ bool key_in_range(int k) { return k >= kKeyMin && k <= kKeyMax; }

// 32-bit mix of the three key fields; any function works, this one is cheap.
__device__ __forceinline__ uint32_t hash_key(int kx, int ky, int kz) {
  uint32_t h = (uint32_t)kx * 0x8DA6B343u + (uint32_t)ky * 0xD8163841u + (uint32_t)kz * 0xCB1AB31Fu;
  return h ^ (h >> 16);
}

// Clamp a float to the int range before conversion, so out-of-range values map
// to out-of-range keys instead of wrapping.
__device__ __forceinline__ int clamp_to_int(float f) {
  f = fminf(fmaxf(f, -2147483520.0f), 2147483520.0f);
  return (int)f;
}

// Exact key of a float32 coordinate.  Fast path: y = x * float(1/r) in float32;
// its error is below |y| * 2^-23, so floor(y) equals floor(x / r) unless y is
// within that distance of an integer; then recompute in binary64.
__device__ __forceinline__ int axis_key_target(float x, float inv_r, double r) {
  float y = x * inv_r;
  float fl = floorf(y);
  float f = y - fl;
  float m = fmaf(fabsf(y), 2.384185791015625e-7f /* 2^-22 */, 2.384185791015625e-7f);
  if (f < m || f > 1.0f - m) {
    double q = __ddiv_rn((double)x, r);
    double k = floor(q);
    k = fmin(fmax(k, -2147483648.0), 2147483647.0);
    return (int)k;
  }
  return clamp_to_int(fl);
}

// Exact sum of float32 values in a double-float (hi + lo) accumulator: TwoSum
// (Knuth; Moeller) keeps hi + lo equal to the running sum as long as the one
// rounding step, lo + e, is exact; that is checked (its own TwoSum error must be
// 0) and reported through `exact`.  While exact, hi + lo is the exact sum, equal
// to the binary64 sum in any order, so no ordering is needed for it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float v, bool& exact) {
  float t, e, u, e2;
  two_sum(hi, v, t, e);
  two_sum(lo, e, u, e2);
  exact = exact && (e2 == 0.0f);
  two_sum(t, u, hi, lo);
}

// Correctly rounded binary64 quotient s / n from the rounded reciprocal and one
// correction step (Markstein's theorem: with y = RN(1/n) and q = RN(s*y), the
// residual r = s - q*n is exact under FMA and RN(q + r*y) = RN(s/n)).
__device__ __forceinline__ double div_rn(double s, double n, double y) {
  const double q = __dmul_rn(s, y);
  const double r = __fma_rn(-q, n, s);
  return __fma_rn(r, y, q);
}

}  // namespace vgicp
