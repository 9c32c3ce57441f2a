// Voxel-map build kernels (arXiv 2202.00242 Sec. III-A: the target cloud is
// discretised into voxels; each voxel aggregates the means and covariances of
// its points).
//
// Pipeline for a batch of maps built from concatenated clouds (one launch per
// step for the whole batch):
//   reset     table slots <- empty: every slot on the first build; afterwards
//             the lookup-table slots the previous build's voxels occupy (the
//             build table is left empty by the scatter)
//   insert    per point: exact key, open-addressing insert (CAS on the 64-bit
//             key, bounded linear probe), count, smallest point index
//   number    first points (the smallest index of their voxel) marked in a
//             bitmap; voxel id = number of first points before the voxel's
//             (a scan of the words' popcounts), so voxels are numbered in order
//             of first appearance, map by map; each first point gives its voxel
//             its count, key and, in the slot, its id
//   sort      per map chunk: the voxels in Morton order of their keys (rank)
//   scan      offsets of the voxels' point lists, in rank order and by voxel
//   scatter   per point: append its index to its voxel's list; the voxel's
//             last point empties its build-table slot
//   capacity  per map: lookup-table capacity from the voxel count
//   finalize  per voxel, in rank order: sort its list, sum means and
//             covariances (exactly, else in binary64 in ascending point index),
//             divide by N, round to float32; copy the points into the voxel-
//             grouped cloud (the lists laid end to end); insert the voxel into
//             its map's lookup table (inline records)
// The result is deterministic and bit-identical to the binary64 definition
// rounded once to float32.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include "vgicp_device.cuh"
#include "vgicp_internal.h"
#include "vgicp_mean.h"

namespace vgicp {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int find_map(const int64_t* __restrict__ off, int32_t n_maps,
                                        int64_t i) {
  // last m with off[m] <= i (empty maps are skipped)
  int lo = 0, hi = n_maps;  // answer in [lo, hi)
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// find_map for the points of one warp, which are consecutive: the first active
// lane searches, the others walk forward from its map (a warp spans few maps).
__device__ __forceinline__ int find_map_warp(const int64_t* __restrict__ off, int32_t n_maps,
                                             int64_t i) {
  const unsigned am = __activemask();
  const int leader = __ffs(am) - 1;
  int m = ((int)(threadIdx.x & 31) == leader) ? find_map(off, n_maps, i) : 0;
  m = __shfl_sync(am, m, leader);
  while (m + 1 < n_maps && __ldg(off + m + 1) <= i) ++m;
  return m;
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

__global__ void init_slots_kernel(Slot* __restrict__ slots, int64_t cap_total) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    Slot e;
    e.key = kEmptyKey;
    e.vid = 0xFFFFFFFFu;
    e.count = 0u;
    slots[s] = e;
  }
}

__global__ void insert_kernel(const float* __restrict__ pts, int64_t n_total,
                              const int64_t* __restrict__ point_off, int32_t n_maps,
                              const int64_t* __restrict__ slot_base,
                              const uint32_t* __restrict__ cap_mask, float inv_r, double r,
                              int32_t max_probe, Slot* slots, uint32_t* __restrict__ pt_slot,
                              int32_t* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int m = find_map_warp(point_off, n_maps, i);
    const int kx = axis_key_target(__ldg(pts + 3 * i + 0), inv_r, r);
    const int ky = axis_key_target(__ldg(pts + 3 * i + 1), inv_r, r);
    const int kz = axis_key_target(__ldg(pts + 3 * i + 2), inv_r, r);
    if (!key_in_range(kx) || !key_in_range(ky) || !key_in_range(kz)) {
      pt_slot[i] = kNoSlot;
      set_status(status, VGICP_ERR_KEY_RANGE);
      continue;
    }
    const unsigned long long key = pack_key(kx, ky, kz);
    const uint32_t mask = __ldg(cap_mask + m);
    const int64_t base = __ldg(slot_base + m);
    uint32_t h = hash_key(kx, ky, kz) & mask;
    uint32_t found = kNoSlot;
    for (int p = 0; p < max_probe; ++p) {
      // one round trip: the CAS either claims an empty slot or returns its key
      const unsigned long long cur = atomicCAS(&slots[base + h].key, kEmptyKey, key);
      if (cur == kEmptyKey || cur == key) {
        found = (uint32_t)(base + h);
        break;
      }
      h = (h + 1) & mask;
    }
    if (found == kNoSlot) {
      pt_slot[i] = kNoSlot;
      set_status(status, VGICP_ERR_HASH_FULL);
      continue;
    }
    atomicAdd(&slots[found].count, 1u);
    atomicMin(&slots[found].vid, (uint32_t)i);
    pt_slot[i] = found;
  }
}



// Rebuild: empty the lookup-table slots the previous build's voxels occupy
// (every slot a build claims belongs to one of its voxels, and spill flags are
// set only on claimed slots), which leaves the tables empty.  (The build table
// is emptied by the scatter of every build.)
__global__ void reset_tables_kernel(int64_t n_max, const uint32_t* __restrict__ n_vox,
                                    const uint32_t* __restrict__ lslot_of, VSlot* vslots) {
  const int64_t V = *n_vox;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V && v < n_max;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t ls = lslot_of[v];
    if (ls != kNoSlot)
      asm volatile("st.global.v8.b32 [%0], {%1, %1, %2, %2, %2, %2, %2, %2};" ::"l"(vslots + ls),
                   "r"(0xFFFFFFFFu), "r"(0u)
                   : "memory");
  }
}



// Per point: append its index to its voxel's list.  The voxel's last point
// (the one whose fill count reaches the voxel's count; every other point of the
// voxel has read the slot before its own increment) empties the build-table
// slot, whose sector it has just read: the build table is empty again when the
// scatter ends, ready for the next build.
__global__ void scatter_kernel(int64_t n_total, const uint32_t* __restrict__ pt_slot, Slot* slots,
                               unsigned long long* bfill, uint32_t* __restrict__ plist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = pt_slot[i];
    if (s == kNoSlot) continue;
    // one read of the slot: voxel id and count
    const uint4 w = *reinterpret_cast<const uint4*>(slots + s);
    const uint32_t v = w.z, c = w.w;
    // (list base << 32 | fill): one atomic gives the point its place
    const unsigned long long bf = atomicAdd(bfill + v, 1ull);
    const uint32_t f = (uint32_t)bf;
    plist[(uint32_t)(bf >> 32) + f] = (uint32_t)i;
    if (f + 1u == c) {
      Slot e;
      e.key = kEmptyKey;
      e.vid = 0xFFFFFFFFu;
      e.count = 0u;
      slots[s] = e;
    }
  }
}

// Inserts voxel v (its key, count, mean and the Cholesky factor of its
// covariance) into its map's lookup table: linear probing from the key's home
// slot, claiming a slot with a CAS on the key; a key placed past its home sets
// the home slot's spill flag.  lslot_of[v] records the slot (kNoSlot if the
// probe limit was reached, which is reported as VGICP_ERR_HASH_FULL).
// lo: the voxel's map.
__device__ __forceinline__ void insert_lookup(uint32_t v, unsigned long long key, uint32_t c,
                                              const float* q, int lo,
                                              const int64_t* __restrict__ slot_base,
                                              const uint32_t* __restrict__ vmask,
                                              int32_t max_probe, VSlot* vslots,
                                              uint32_t* __restrict__ lslot_of, int32_t* status) {
  const unsigned long long fm = (1ull << kKeyBits) - 1ull;
  const int kx = (int)((key >> (2 * kKeyBits)) & fm) - kKeyBias;
  const int ky = (int)((key >> kKeyBits) & fm) - kKeyBias;
  const int kz = (int)(key & fm) - kKeyBias;
  const uint32_t mask = vmask[lo];
  VSlot* t = vslots + slot_base[lo];
  const uint32_t home = hash_key(kx, ky, kz) & mask;
  uint32_t h = home;
  bool placed = false;
  for (int p = 0; p < max_probe; ++p) {
    if (atomicCAS(&t[h].key, kEmptyKey, key) == kEmptyKey) {
      placed = true;
      break;
    }
    h = (h + 1) & mask;
  }
  if (placed && h != home) atomicOr(&t[home].spill, 1u);
  lslot_of[v] = placed ? (uint32_t)(slot_base[lo] + h) : kNoSlot;
  if (!placed) {
    set_status(status, VGICP_ERR_HASH_FULL);
    return;
  }
  VSlot& sl = t[h];
  sl.vid = v;
  sl.count = c;
  sl.mu[0] = q[0];
  sl.mu[1] = q[1];
  sl.mu[2] = q[2];
  // the Cholesky factor L of C' (the linearization forms R^T C' R as (R^T L)(R^T L)^T);
  // a non-positive pivot (a semi-definite C') leaves its column zero
  const float l00 = q[3] > 0.f ? sqrtf(q[3]) : 0.f;
  const float il0 = l00 > 0.f ? 1.0f / l00 : 0.f;
  const float l10 = q[4] * il0, l20 = q[5] * il0;
  const float p11 = q[6] - l10 * l10;
  const float l11 = p11 > 0.f ? sqrtf(p11) : 0.f;
  const float l21 = l11 > 0.f ? (q[7] - l20 * l10) / l11 : 0.f;
  const float p22 = q[8] - l20 * l20 - l21 * l21;
  const float l22 = p22 > 0.f ? sqrtf(p22) : 0.f;
  sl.cov[0] = l00;
  sl.cov[1] = l10;
  sl.cov[2] = l20;
  sl.cov[3] = l11;
  sl.cov[4] = l21;
  sl.cov[5] = l22;
  sl.pad1[0] = 0.0f;
  sl.pad1[1] = 0.0f;
}

// Per-voxel sums and the grouped cloud.  A CTA takes 128 consecutive ranks,
// whose point lists are one contiguous segment of plist:
//   1. the segment is loaded into shared memory (coalesced) and each thread
//      sorts its voxel's short list there by point index (segments longer than
//      the staging buffer sort in place in global memory);
//   2. point-parallel: every thread gathers points of the segment and writes
//      them to the grouped cloud at their list positions (balanced, coalesced
//      writes; the random reads all in flight at once);
//   3. voxel-parallel: each thread sums its voxel's points from the grouped copy
//      just written (L2-resident) and writes the voxel record.
constexpr int kFinThreads = 128;
constexpr int kFinStage = 3072;  // indices staged per CTA

__device__ __forceinline__ void insertion_sort(uint32_t* L, uint32_t c) {
  for (uint32_t a = 1; a < c; ++a) {
    const uint32_t x = L[a];
    int b = (int)a - 1;
    while (b >= 0 && L[b] > x) {
      L[b + 1] = L[b];
      --b;
    }
    L[b + 1] = x;
  }
}

// Map of rank (or voxel id) r: the last m with vbase[m] <= r.
__device__ __forceinline__ int map_of_rank(const uint32_t* __restrict__ vbase, int32_t n_maps,
                                           int64_t r) {
  int lo = 0, hi = n_maps;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)vbase[mid] <= r) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kFinThreads) finalize_kernel(
    int64_t n_max, const uint32_t* __restrict__ n_vox, const uint32_t* __restrict__ n_valid,
    const float* __restrict__ pts, const float* __restrict__ covs,
    const uint32_t* __restrict__ vorder, const uint32_t* __restrict__ goff,
    uint32_t* __restrict__ plist, float4* __restrict__ recs, float* gpts, float* gcovs,
    const unsigned long long* __restrict__ vkeys, int32_t n_maps,
    const uint32_t* __restrict__ vbase, const int64_t* __restrict__ slot_base,
    const uint32_t* __restrict__ vmask, int32_t max_probe, VSlot* vslots,
    uint32_t* __restrict__ lslot_of, int32_t* status) {
  __shared__ uint32_t stage[kFinStage];
  __shared__ int seg_map[2];
  const int64_t V = min((int64_t)*n_vox, n_max);
  const uint32_t total = *n_valid;  // end of the last list (goff[V] is not stored)
  for (int64_t r0 = (int64_t)blockIdx.x * kFinThreads; r0 < V; r0 += (int64_t)gridDim.x * kFinThreads) {
    const int64_t r1 = min(V, r0 + kFinThreads);
    // list bounds from consecutive offsets: no dependent load through vorder
    const uint32_t seg0 = goff[r0];
    const uint32_t seg1 = r1 < V ? goff[r1] : total;
    const uint32_t len = seg1 - seg0;
    const bool staged = len <= (uint32_t)kFinStage;
    const int64_t r = r0 + threadIdx.x;
    const bool mine = r < r1;
    if (threadIdx.x == 0) {  // the maps of the CTA's first and last ranks
      seg_map[0] = map_of_rank(vbase, n_maps, r0);
      seg_map[1] = map_of_rank(vbase, n_maps, r1 - 1);
    }
    const uint32_t v = mine ? vorder[r] : 0u;
    const uint32_t o = mine ? goff[r] : 0u;
    const uint32_t c = mine ? (r + 1 < V ? goff[r + 1] : total) - o : 0u;
    // 1. sort the lists by point index
    if (staged) {
      for (uint32_t i = threadIdx.x; i < len; i += kFinThreads) stage[i] = plist[seg0 + i];
      __syncthreads();
      if (mine) insertion_sort(stage + (o - seg0), c);
    } else if (mine) {
      insertion_sort(plist + o, c);
    }
    __syncthreads();
    // 2. gather into the grouped cloud
    const uint32_t* lst = staged ? stage : plist + seg0;
    for (uint32_t i = threadIdx.x; i < len; i += kFinThreads) {
      const int64_t j = lst[i];
      const float x = __ldg(pts + 3 * j), y = __ldg(pts + 3 * j + 1), z = __ldg(pts + 3 * j + 2);
      const float2* cv = reinterpret_cast<const float2*>(covs + 6 * j);
      const float2 c0 = __ldg(cv), c1 = __ldg(cv + 1), c2 = __ldg(cv + 2);
      const int64_t d = (int64_t)seg0 + i;
      gpts[3 * d + 0] = x;
      gpts[3 * d + 1] = y;
      gpts[3 * d + 2] = z;
      float2* gc = reinterpret_cast<float2*>(gcovs + 6 * d);
      gc[0] = c0;
      gc[1] = c1;
      gc[2] = c2;
    }
    __syncthreads();  // the CTA's global writes are visible to the CTA after this
    // 3. sums from the grouped copy (plain loads: written by this kernel)
    if (mine) {
      float hi[9], lo[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) hi[k] = lo[k] = 0.0f;
      bool exact = true;
      for (uint32_t a = 0; a < c; ++a) {
        const int64_t d = (int64_t)o + a;
        float f[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) f[k] = gpts[3 * d + k];
        const float2* gc = reinterpret_cast<const float2*>(gcovs + 6 * d);
        const float2 c0 = gc[0], c1 = gc[1], c2 = gc[2];
        f[3] = c0.x; f[4] = c0.y; f[5] = c1.x; f[6] = c1.y; f[7] = c2.x; f[8] = c2.y;
        // hi + lo stays the exact sum while each TwoSum error adds exactly to lo
        // (checked); renormalised once at the end
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          float t, e, u, e2;
          two_sum(hi[k], f[k], t, e);
          two_sum(lo[k], e, u, e2);
          exact = exact && (e2 == 0.0f);
          hi[k] = t;
          lo[k] = u;
        }
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {  // hi = RN(hi + lo), lo = the exact remainder
        float t, e;
        two_sum(hi[k], lo[k], t, e);
        hi[k] = t;
        lo[k] = e;
      }
      // q = RN32(RN64(sum / N)) per component: from the exact float pair in
      // float32 where certified, else (rare) from the binary64 definition
      float q[9];
      uint32_t need64 = exact ? 0u : 0x1FFu;
      if (exact) {
        const float rN = __frcp_rn((float)c);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          bool ok;
          q[k] = mean_rn32(hi[k], lo[k], c, rN, ok);
          if (!ok) need64 |= 1u << k;
        }
      }
      if (need64) {
        double sum[9];
        if (exact) {
#pragma unroll
          for (int k = 0; k < 9; ++k) sum[k] = __dadd_rn((double)hi[k], (double)lo[k]);  // exact
        } else {
          // binary64 sum in ascending point index (the grouped order; rare: large
          // dynamic range)
#pragma unroll
          for (int k = 0; k < 9; ++k) sum[k] = 0.0;
          for (uint32_t a = 0; a < c; ++a) {
            const int64_t d = (int64_t)o + a;
#pragma unroll
            for (int k = 0; k < 3; ++k) sum[k] = __dadd_rn(sum[k], (double)gpts[3 * d + k]);
#pragma unroll
            for (int k = 0; k < 6; ++k) sum[3 + k] = __dadd_rn(sum[3 + k], (double)gcovs[6 * d + k]);
          }
        }
        const double N = (double)c;
        const double y = __drcp_rn(N);
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (need64 & (1u << k)) q[k] = __double2float_rn(div_rn(sum[k], N, y));
      }
      recs[3 * v + 0] = make_float4(q[0], q[1], q[2], __uint_as_float(c));
      recs[3 * v + 1] = make_float4(q[3], q[4], q[5], q[6]);
      recs[3 * v + 2] = make_float4(q[7], q[8], 0.0f, 0.0f);
      // the voxel's map (ranks and voxel ids of a map share its range
      // [vbase[m], vbase[m + 1])): a CTA's ranks rarely span two maps
      int m = seg_map[0];
      while (m < seg_map[1] && (int64_t)vbase[m + 1] <= r) ++m;
      insert_lookup(v, vkeys[v], c, q, m, slot_base, vmask, max_probe, vslots,
                    lslot_of, status);
    }
    __syncthreads();  // the stage is reused by the next batch
  }
}

// 10 bits per axis of the key, interleaved (a locality order, not a unique code).
__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  x &= 1023u;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}
__device__ __forceinline__ uint32_t morton_of_key(unsigned long long key) {
  const unsigned long long fm = (1ull << kKeyBits) - 1ull;
  const uint32_t kx = (uint32_t)((key >> (2 * kKeyBits)) & fm);
  const uint32_t ky = (uint32_t)((key >> kKeyBits) & fm);
  const uint32_t kz = (uint32_t)(key & fm);
  return spread10(kx) | (spread10(ky) << 1) | (spread10(kz) << 2);
}

// One CTA per (map, chunk): bitonic sort of the chunk's voxels by Morton code in
// shared memory (ties by voxel id); vorder[rank] = v and gcount[rank] = the
// voxel's point count.
//
// Element i lives at i + i / 16 (one pad word per 16), which keeps every access
// pattern below free of bank conflicts.  Each pass loads a group of up to 16
// elements per thread into registers and applies up to four consecutive stages
// of the network there: a group is the elements i0 + t s (t < 2^M), closed under
// the strides s .. s 2^(M-1), so a merge level of stride 2^(p-1) .. 1 takes
// ceil(p / 4) passes through shared memory instead of p.
constexpr int kSortThreads = 1024;
constexpr int kSortSmemElems = kMortonChunk + kMortonChunk / 16;

__device__ __forceinline__ uint32_t sort_phys(uint32_t i) { return i + (i >> 4); }

__device__ __forceinline__ void cmp_swap(unsigned long long& a, unsigned long long& b, bool up) {
  if ((a > b) == up) {
    const unsigned long long t = a;
    a = b;
    b = t;
  }
}

// The stages of strides s 2^(M-1) .. s of merge level k on every group.
template <int M>
__device__ __forceinline__ void bitonic_pass(unsigned long long* sk, uint32_t N, uint32_t k,
                                             uint32_t s_log) {
  constexpr int G = 1 << M;
  const uint32_t s = 1u << s_log;
  for (uint32_t g = threadIdx.x; g < (N >> M); g += blockDim.x) {
    const uint32_t i0 = ((g >> s_log) << (s_log + M)) | (g & (s - 1u));
    const bool up = (i0 & k) == 0u;  // the same for the whole group (its bits are below k)
    unsigned long long r[G];
#pragma unroll
    for (int t = 0; t < G; ++t) r[t] = sk[sort_phys(i0 + (uint32_t)t * s)];
#pragma unroll
    for (int j = G >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int t = 0; t < G; ++t)
        if ((t ^ j) > t) cmp_swap(r[t], r[t ^ j], up);
#pragma unroll
    for (int t = 0; t < G; ++t) sk[sort_phys(i0 + (uint32_t)t * s)] = r[t];
  }
}

__global__ void __launch_bounds__(kSortThreads) morton_sort_kernel(
    const int2* __restrict__ chunks, const uint32_t* __restrict__ vbase,
    const unsigned long long* __restrict__ vkeys, const uint32_t* __restrict__ vcount,
    uint32_t* __restrict__ vorder, uint32_t* __restrict__ gcount) {
  extern __shared__ unsigned long long sk[];
  const int m = chunks[blockIdx.x].x;
  const uint32_t V = vbase[m + 1] - vbase[m];
  const uint32_t lo = (uint32_t)chunks[blockIdx.x].y * kMortonChunk;
  if (lo >= V) return;
  const uint32_t cnt = min((uint32_t)kMortonChunk, V - lo);
#ifdef VGICP_NO_MORTON
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    vorder[vbase[m] + lo + i] = vbase[m] + lo + i;
    gcount[vbase[m] + lo + i] = vcount[vbase[m] + lo + i];
  }
  return;
#endif
  uint32_t N = 16;  // at least one full register group
  while (N < cnt) N <<= 1;
  const uint32_t first = vbase[m] + lo;
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
    sk[sort_phys(i)] =
        i < cnt ? (((unsigned long long)morton_of_key(vkeys[first + i]) << 32) | i) : ~0ull;
  __syncthreads();
  // levels k = 2 .. 16: inside blocks of 16 consecutive elements
  for (uint32_t g = threadIdx.x; g < (N >> 4); g += blockDim.x) {
    unsigned long long r[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) r[t] = sk[sort_phys(16u * g + t)];
#pragma unroll
    for (int k = 2; k <= 16; k <<= 1)
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if ((t ^ j) > t) cmp_swap(r[t], r[t ^ j], ((16u * g + t) & (uint32_t)k) == 0u);
#pragma unroll
    for (int t = 0; t < 16; ++t) sk[sort_phys(16u * g + t)] = r[t];
  }
  __syncthreads();
  // levels k = 32 .. N: strides 2^(p-1) .. 1 in passes of up to four, the
  // partial pass (p mod 4 strides) first
  for (uint32_t p = 5; (1u << p) <= N; ++p) {
    const uint32_t k = 1u << p;
    int top = (int)p - 1;  // log2 of the largest stride not yet applied
    const int rem = (int)(p & 3u);
    if (rem) {
      const uint32_t s_log = (uint32_t)(top - rem + 1);
      if (rem == 1) bitonic_pass<1>(sk, N, k, s_log);
      else if (rem == 2) bitonic_pass<2>(sk, N, k, s_log);
      else bitonic_pass<3>(sk, N, k, s_log);
      top -= rem;
      __syncthreads();
    }
    for (; top >= 0; top -= 4) {
      bitonic_pass<4>(sk, N, k, (uint32_t)(top - 3));
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const uint32_t v = first + (uint32_t)(sk[sort_phys(i)] & 0xFFFFFFFFull);
    vorder[first + i] = v;
    gcount[first + i] = vcount[v];
  }
}



__device__ __forceinline__ uint32_t lookup_capacity(uint32_t nvox) {
  uint32_t c = 16;
  while (c < kLookupLoad * nvox) c <<= 1;
  return c;
}

// Per map (blockIdx.y): lookup-table capacity from its voxel count; with
// clear_all, every slot of the map's region emptied (the first build, whose
// region is fresh; later builds find the region empty after the reset).
__global__ void vslot_init_kernel(const int64_t* __restrict__ slot_base,
                                  const uint32_t* __restrict__ vbase, VSlot* vslots,
                                  uint32_t* __restrict__ vmask, int32_t clear_all) {
  const int m = blockIdx.y;
  // the region was sized by the first build; a rebuild with more voxels runs at a
  // higher load factor (an insertion past max_probe reports VGICP_ERR_HASH_FULL)
  const uint32_t region = (uint32_t)(slot_base[m + 1] - slot_base[m]);
  const uint32_t cap = min(lookup_capacity(vbase[m + 1] - vbase[m]), region);
  if (clear_all) {
    VSlot* t = vslots + slot_base[m];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < region;
         i += gridDim.x * blockDim.x) {
      // the whole first 32-B sector (key = empty, spill = 0): no read-modify-write
      asm volatile("st.global.v8.b32 [%0], {%1, %1, %2, %2, %2, %2, %2, %2};" ::"l"(t + i),
                   "r"(0xFFFFFFFFu), "r"(0u)
                   : "memory");
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) vmask[m] = cap - 1u;
}

// ---- exclusive scan of uint32 (three phases) --------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanTile = kScanThreads * kScanPerThread;

__device__ __forceinline__ int64_t scan_len(int64_t n_max, const uint32_t* n_dev) {
  return n_dev ? min(n_max, (int64_t)*n_dev) : n_max;
}

// Block-wide exclusive scan of one value per thread (T threads); returns the
// thread's exclusive prefix and writes the block total to *total.
template <int T>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t x, uint32_t* total) {
  static_assert(T % 32 == 0 && T <= 1024, "block size");
  __shared__ uint32_t warp_sum[T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sum[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t ws = lane < T / 32 ? warp_sum[lane] : 0u;
    uint32_t wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < T / 32) warp_sum[lane] = wi - ws;
    if (lane == T / 32 - 1) *total = wi;
  }
  __syncthreads();
  uint32_t r = warp_sum[w] + inc - x;
  __syncthreads();
  return r;
}

__global__ void scan_tile_sums_kernel(const uint32_t* __restrict__ in, int64_t n_max,
                                      const uint32_t* n_dev, uint32_t* __restrict__ sums) {
  const int64_t n = scan_len(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k)
    if (base + k < n) s += in[base + k];
  __shared__ uint32_t total;
  block_exclusive<kScanThreads>(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One CTA: each thread scans a contiguous run of the tile sums.
constexpr int kScanSumsThreads = 1024;
__global__ void __launch_bounds__(kScanSumsThreads) scan_sums_kernel(
    uint32_t* __restrict__ sums, int64_t nb, uint32_t* __restrict__ total_dev) {
  __shared__ uint32_t total;
  const int64_t per = (nb + kScanSumsThreads - 1) / kScanSumsThreads;
  const int64_t a = min(nb, (int64_t)threadIdx.x * per), b = min(nb, a + per);
  uint32_t s = 0;
  for (int64_t i = a; i < b; ++i) s += sums[i];
  uint32_t run = block_exclusive<kScanSumsThreads>(s, &total);
  for (int64_t i = a; i < b; ++i) {
    const uint32_t x = sums[i];
    sums[i] = run;
    run += x;
  }
  if (threadIdx.x == 0 && total_dev) *total_dev = total;
}

__global__ void scan_tiles_kernel(const uint32_t* in, uint32_t* out, int64_t n_max,
                                  const uint32_t* n_dev, const uint32_t* __restrict__ sums) {
  const int64_t n = scan_len(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t v[kScanPerThread];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  __shared__ uint32_t total;
  uint32_t run = block_exclusive<kScanThreads>(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

// Last pass of the scan of the rank-ordered counts: goff[r] = the offset of rank
// r's list, also stored by voxel for the scatter, as (base << 32 | fill 0).
__global__ void scan_lists_kernel(const uint32_t* __restrict__ gcount, uint32_t* __restrict__ goff,
                                  int64_t n_max, const uint32_t* __restrict__ n_dev,
                                  const uint32_t* __restrict__ sums,
                                  const uint32_t* __restrict__ vorder,
                                  unsigned long long* __restrict__ bfill) {
  const int64_t n = scan_len(n_max, n_dev);
  const int64_t b0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPerThread;
  uint32_t v[kScanPerThread];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    v[k] = (b0 + k < n) ? gcount[b0 + k] : 0u;
    s += v[k];
  }
  __shared__ uint32_t total;
  uint32_t run = block_exclusive<kScanThreads>(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    if (b0 + k < n) {
      goff[b0 + k] = run;
      bfill[vorder[b0 + k]] = (unsigned long long)run << 32;  // fill 0
    }
    run += v[k];
  }
}

// ---- first-appearance numbering -----------------------------------------
// A point is its voxel's first if its index is the smallest of the voxel (the
// build-table slot holds that index after the insert).  The first points are
// marked in a bitmap (one warp ballot per 32 points); a voxel's id is the number
// of marked points before its first point (an exclusive scan of the words'
// popcounts), so voxels are numbered in order of first appearance, map by map.

// One thread per point; every warp is whole (the grid covers n rounded up to
// 32), so the ballot sees all 32 lanes.
__global__ void first_bits_kernel(const uint32_t* __restrict__ pt_slot,
                                  const Slot* __restrict__ slots, int64_t n,
                                  uint32_t* __restrict__ bitmap) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool f = false;
  if (i < n) {
    const uint32_t ps = pt_slot[i];
    f = ps != kNoSlot && slots[ps].vid == (uint32_t)i;
  }
  const unsigned b = __ballot_sync(0xFFFFFFFFu, f);
  if ((threadIdx.x & 31) == 0 && i < n) bitmap[i >> 5] = b;
}

__global__ void popc_words_kernel(const uint32_t* __restrict__ bitmap, int64_t n_words,
                                  uint32_t* __restrict__ out) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_words;
       w += (int64_t)gridDim.x * blockDim.x)
    out[w] = (uint32_t)__popc(bitmap[w]);
}

// Number of first points before point i (wscan: the exclusive scan of the words'
// popcounts; the word of index n exists and has no bit at or above n).
__device__ __forceinline__ uint32_t first_rank(const uint32_t* __restrict__ bitmap,
                                               const uint32_t* __restrict__ wscan, uint32_t i) {
  const uint32_t w = i >> 5;
  return wscan[w] + (uint32_t)__popc(bitmap[w] & ((1u << (i & 31u)) - 1u));
}

// Each first point gives its voxel its id: the voxel's count and key are
// recorded by id and the id replaces the index in the build-table slot.
__global__ void assign_ids_kernel(const uint32_t* __restrict__ bitmap,
                                  const uint32_t* __restrict__ wscan, int64_t n,
                                  const uint32_t* __restrict__ pt_slot, Slot* slots,
                                  uint32_t* __restrict__ vcount,
                                  unsigned long long* __restrict__ vkeys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!((bitmap[i >> 5] >> (i & 31)) & 1u)) continue;
    const uint32_t id = first_rank(bitmap, wscan, (uint32_t)i);
    Slot* sl = slots + pt_slot[i];
    vcount[id] = sl->count;
    vkeys[id] = sl->key;
    sl->vid = id;
  }
}

// vbase[m] = voxels of the maps before m; vbase[n_maps] and *n_vox = all.
__global__ void vbase_kernel(int32_t n_maps, int64_t n_total, const int64_t* __restrict__ point_off,
                             const uint32_t* __restrict__ bitmap,
                             const uint32_t* __restrict__ wscan, uint32_t* __restrict__ vbase,
                             uint32_t* __restrict__ n_vox) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > n_maps) return;
  const int64_t o = m < n_maps ? point_off[m] : n_total;
  const uint32_t v = first_rank(bitmap, wscan, (uint32_t)o);
  vbase[m] = v;
  if (m == n_maps) *n_vox = v;
}

// One thread per element (no grid-stride cap): CTAs are dispatched roughly in
// index order, so the maps being worked on at any moment are a few consecutive
// ones whose clouds and tables stay in L2 while their random accesses land.
int grid_for(int64_t n, int threads) {
  const int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 0x7FFFFFFF));
}

}  // namespace

size_t scan_tmp_elems(int64_t n_max) { return (size_t)((n_max + kScanTile - 1) / kScanTile) + 1; }

int launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n_max, const uint32_t* n_dev,
                          uint32_t* block_tmp, uint32_t* total_dev, cudaStream_t st) {
  if (n_max <= 0) {
    if (total_dev) VGICP_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), st));
    return VGICP_OK;
  }
  const int64_t nb = (n_max + kScanTile - 1) / kScanTile;
  scan_tile_sums_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n_max, n_dev, block_tmp);
  scan_sums_kernel<<<1, kScanSumsThreads, 0, st>>>(block_tmp, nb, total_dev);
  scan_tiles_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n_max, n_dev, block_tmp);
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(3);
  return VGICP_OK;
}

// First build of a set: reads the per-map voxel counts back (one stream
// synchronization) and allocates each map's lookup-table region at
// next_pow2(max(16, kLookupLoad V, 2 n)) slots; a build uses
// min(next_pow2(kLookupLoad V), region) of it.
int size_lookup_tables(MapSet* s, cudaStream_t st) {
  std::vector<uint32_t> vb((size_t)s->n_maps + 1);
  VGICP_CUDA_TRY(cudaMemcpyAsync(vb.data(), s->d_vbase, sizeof(uint32_t) * vb.size(),
                                 cudaMemcpyDeviceToHost, st));
  VGICP_CUDA_TRY(cudaStreamSynchronize(st));
  s->vslot_base.assign((size_t)s->n_maps + 1, 0);
  int64_t total = 0;
  for (int32_t m = 0; m < s->n_maps; ++m) {
    const uint64_t V = vb[m + 1] >= vb[m] ? vb[m + 1] - vb[m] : 0;
    // at least 2 n slots, so that a rebuild with up to V = n voxels still fits
    // (load factor <= 1/2); the first build's capacity next_pow2(kLookupLoad V)
    // when larger
    const uint64_t nm = (uint64_t)(s->point_off[m + 1] - s->point_off[m]);
    uint64_t c = 16;
    while (c < kLookupLoad * V || c < 2 * nm) c <<= 1;
    s->vslot_base[m] = total;
    total += (int64_t)c;
  }
  s->vslot_base[s->n_maps] = total;
  if (total >= (int64_t)0xFFFFFFFFll)
    return set_error(VGICP_ERR_INVALID_ARG, "more than 2^32-1 lookup slots in one batch");
  cudaError_t e = device_malloc(&s->d_vblock, sizeof(VSlot) * (size_t)total, nullptr, false);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->d_vblock = nullptr;
    return set_error(VGICP_ERR_OOM, "lookup table allocation of " +
                                        std::to_string(sizeof(VSlot) * (size_t)total) +
                                        " bytes failed");
  }
  s->d_vslots = static_cast<VSlot*>(s->d_vblock);
  s->vcap_total = total;
  VGICP_CUDA_TRY(cudaMemcpy(s->d_vslot_base, s->vslot_base.data(),
                            sizeof(int64_t) * s->vslot_base.size(), cudaMemcpyHostToDevice));
  return VGICP_OK;
}

int launch_build(MapSet* s, const float* points, const float* covs, cudaStream_t st) {
  const int64_t n = s->n_total;
  // light kernels over voxels (V <= n is on the device): grid-stride, capped grid
  const int gv = std::min<int>(grid_for(std::max<int64_t>(n, 1), kThreads), device_sm_count() * 8);
  // was_built: the tables hold only the previous build's voxels (a build that
  // stops on an error leaves `built` cleared, so the next one starts over)
  const bool was_built = s->built;
  s->built = false;
  if (was_built) {
    // empty the slots of the previous build's voxels
    reset_tables_kernel<<<gv, kThreads, 0, st>>>(n, s->d_num_voxels, s->d_lslot_of,
                                                 s->d_vslots);
    count_launches(1);
  } else if (s->cap_total > 0) {
    init_slots_kernel<<<grid_for(s->cap_total, kThreads), kThreads, 0, st>>>(s->d_slots,
                                                                          s->cap_total);
    count_launches(1);
  }
  VGICP_CUDA_TRY(cudaMemsetAsync(s->d_status, 0, sizeof(int32_t), st));
  if (n == 0) {
    VGICP_CUDA_TRY(cudaMemsetAsync(s->d_num_voxels, 0, sizeof(uint32_t), st));
    VGICP_CUDA_TRY(cudaMemsetAsync(s->d_vbase, 0, sizeof(uint32_t) * (s->n_maps + 1), st));
    if (!s->d_vblock) {
      const int rc = size_lookup_tables(s, st);
      if (rc != VGICP_OK) return rc;
    }
    vslot_init_kernel<<<dim3(1, s->n_maps), kThreads, 0, st>>>(s->d_vslot_base, s->d_vbase,
                                                              s->d_vslots, s->d_vmask,
                                                              was_built ? 0 : 1);
    VGICP_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    s->built = true;
    return VGICP_OK;
  }
  const float inv_r = (float)(1.0 / s->resolution);
  const int g = grid_for(n, kThreads);
  insert_kernel<<<g, kThreads, 0, st>>>(points, n, s->d_point_off, s->n_maps, s->d_slot_base,
                                        s->d_cap_mask, inv_r, s->resolution, s->max_probe,
                                        s->d_slots, s->d_pt_slot, s->d_status);
  // voxel ids in order of first appearance: first points marked in d_flag, the
  // words' popcounts scanned in d_vfill (both dead afterwards)
  int rc = VGICP_OK;
  {
    const int64_t n_words = n / 32 + 1;
    uint32_t* bitmap = s->d_flag;
    uint32_t* wscan = s->d_vfill;
    VGICP_CUDA_TRY(cudaMemsetAsync(bitmap + n / 32, 0, sizeof(uint32_t), st));
    first_bits_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(s->d_pt_slot, s->d_slots, n,
                                                                  bitmap);
    popc_words_kernel<<<grid_for(n_words, kThreads), kThreads, 0, st>>>(bitmap, n_words, wscan);
    rc = launch_exclusive_scan(wscan, wscan, n_words, nullptr, s->d_scan_tmp, nullptr, st);
    if (rc != VGICP_OK) return rc;
    assign_ids_kernel<<<g, kThreads, 0, st>>>(bitmap, wscan, n, s->d_pt_slot, s->d_slots,
                                              s->d_vcount, s->d_vkeys);
    vbase_kernel<<<(s->n_maps + 1 + 127) / 128, 128, 0, st>>>(s->n_maps, n, s->d_point_off,
                                                              bitmap, wscan, s->d_vbase,
                                                              s->d_num_voxels);
    VGICP_CUDA_TRY(cudaGetLastError());
    count_launches(4);
  }
  if (!s->d_vblock) {
    rc = size_lookup_tables(s, st);
    if (rc != VGICP_OK) return rc;
  }
  // Morton order of the voxels (chunks of a map), the list offsets in that order,
  // the lists, then the per-voxel sums (which also write the grouped clouds).
  // d_vfill (the numbering's word scan) is dead after the id assignment.
  uint32_t* vorder = s->d_voff;
  uint32_t* gcount = s->d_vfill;
  // the lists' (base << 32 | fill) words, by voxel: in the record storage, which
  // finalize fills only after the scatter (8 of its 48 B per voxel)
  unsigned long long* bfill = reinterpret_cast<unsigned long long*>(s->d_recs);
  {
    // the sort's shared memory is above the default limit: opt in once per device
    static std::mutex attr_mu;
    static bool attr_set[kMaxDevices] = {false};
    int dev = 0;
    VGICP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
      return set_error(VGICP_ERR_INVALID_ARG, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(attr_mu);
    if (!attr_set[dev]) {
      VGICP_CUDA_TRY(cudaFuncSetAttribute(morton_sort_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(unsigned long long) * kSortSmemElems)));
      attr_set[dev] = true;
    }
  }
  morton_sort_kernel<<<s->n_chunks, kSortThreads, sizeof(unsigned long long) * kSortSmemElems,
                       st>>>(s->d_chunks, s->d_vbase, s->d_vkeys, s->d_vcount, vorder, gcount);
  VGICP_CUDA_TRY(cudaGetLastError());
  // list offsets in rank order, and by voxel
  {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    scan_tile_sums_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(gcount, n, s->d_num_voxels,
                                                                 s->d_scan_tmp);
    scan_sums_kernel<<<1, kScanSumsThreads, 0, st>>>(s->d_scan_tmp, nb, s->d_num_valid);
    scan_lists_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(gcount, s->d_goff, n,
                                                             s->d_num_voxels, s->d_scan_tmp,
                                                             vorder, bfill);
    VGICP_CUDA_TRY(cudaGetLastError());
    count_launches(3);
  }
  scatter_kernel<<<g, kThreads, 0, st>>>(n, s->d_pt_slot, s->d_slots, bfill, s->d_plist);
  int64_t max_cap = 16;
  for (int32_t m = 0; m < s->n_maps; ++m)
    max_cap = std::max<int64_t>(max_cap, s->vslot_base[m + 1] - s->vslot_base[m]);
  // the first build empties the whole lookup region; later ones set the masks only
  const unsigned gx =
      was_built ? 1u : (unsigned)std::min<int64_t>(64, (max_cap + kThreads - 1) / kThreads);
  vslot_init_kernel<<<dim3(gx, s->n_maps), kThreads, 0, st>>>(s->d_vslot_base, s->d_vbase,
                                                             s->d_vslots, s->d_vmask,
                                                             was_built ? 0 : 1);
  // sums, records, grouped clouds and the lookup tables
  finalize_kernel<<<g, kFinThreads, 0, st>>>(
      n, s->d_num_voxels, s->d_num_valid, points, covs, vorder, s->d_goff, s->d_plist, s->d_recs,
      s->d_gpts, s->d_gcovs, s->d_vkeys, s->n_maps, s->d_vbase, s->d_vslot_base, s->d_vmask,
      s->max_probe, s->d_vslots, s->d_lslot_of, s->d_status);
  VGICP_CUDA_TRY(cudaGetLastError());
  // insert, sort, scatter, vslot init, finalize (+ reset or init: 1; numbering: 4;
  // the two scans: 3 each)
  count_launches(5);
  s->built = true;
  return VGICP_OK;
}

}  // namespace vgicp
