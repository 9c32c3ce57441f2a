// Voxel-grid downsampling with timestamp averaging (arXiv 2202.00242 Sec. III-C:
// the input clouds are downsampled by a voxel grid; each voxel averages the
// timestamps of its points as well as their positions, and a point whose time
// lies far from its voxel's is put in another, new voxel so that the first and
// last points of a scan are not fused).
//
// Reading (deterministic): a point's voxel is floor(p / r) (binary64
// semantics); the voxel's reference time is that of its first point in index
// order; a point more than `split` away from it in time goes to the voxel's
// second output voxel.  Output voxels are numbered in order of first
// appearance, cloud by cloud; each holds the mean of its points' positions and
// times, the binary64 mean rounded to float32 (exact double-float sums, else
// binary64 sums in index order).
//
//   insert   per point: exact key, CAS into the cloud's table, first index
//   group    per point: sub-voxel from the first point's time; first index of
//            each (voxel, sub) group
//   scan     output ids in first-appearance order
//   count, scan, scatter: the points of each output voxel, contiguous
//   finalize per output voxel: sort its list, exact sums, means
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "vgicp.h"
#include "vgicp_device.cuh"
#include "vgicp_internal.h"

namespace vgicp {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxProbe = 64;
constexpr uint32_t kNone = 0xFFFFFFFFu;

struct __align__(16) DsSlot {
  unsigned long long key;
  uint32_t first;  // smallest point index (global) in the cell
  uint32_t pad;
};

__device__ __forceinline__ int cloud_of(const int64_t* __restrict__ off, int32_t n, int64_t i) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

#define DS_LOOP(i, n)                                                         \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

__global__ void ds_init_kernel(DsSlot* slots, int64_t cap, uint32_t* gfirst) {
  DS_LOOP(s, cap) {
    DsSlot e;
    e.key = kEmptyKey;
    e.first = kNone;
    e.pad = 0u;
    slots[s] = e;
    gfirst[2 * s] = kNone;
    gfirst[2 * s + 1] = kNone;
  }
}

__global__ void ds_insert_kernel(const float* __restrict__ pts, int64_t n,
                                 const int64_t* __restrict__ off, int32_t n_clouds, float inv_r,
                                 double r, const int64_t* __restrict__ base,
                                 const uint32_t* __restrict__ mask, DsSlot* slots,
                                 uint32_t* __restrict__ pt_slot, int32_t* status) {
  DS_LOOP(i, n) {
    const int c = cloud_of(off, n_clouds, i);
    const int kx = axis_key_target(pts[3 * i], inv_r, r);
    const int ky = axis_key_target(pts[3 * i + 1], inv_r, r);
    const int kz = axis_key_target(pts[3 * i + 2], inv_r, r);
    if (!key_in_range(kx) || !key_in_range(ky) || !key_in_range(kz)) {
      pt_slot[i] = kNone;
      set_status(status, VGICP_ERR_KEY_RANGE);
      continue;
    }
    const unsigned long long key = pack_key(kx, ky, kz);
    DsSlot* t = slots + base[c];
    const uint32_t m = mask[c];
    uint32_t h = hash_key(kx, ky, kz) & m;
    uint32_t found = kNone;
    for (int p = 0; p < kMaxProbe; ++p) {
      unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(&t[h].key);
      if (cur == kEmptyKey) {
        cur = atomicCAS(&t[h].key, kEmptyKey, key);
        if (cur == kEmptyKey) cur = key;
      }
      if (cur == key) {
        found = h;
        break;
      }
      h = (h + 1) & m;
    }
    if (found == kNone) {
      pt_slot[i] = kNone;
      set_status(status, VGICP_ERR_HASH_FULL);
      continue;
    }
    atomicMin(&t[found].first, (uint32_t)i);
    pt_slot[i] = (uint32_t)(base[c] + found);
  }
}

__global__ void ds_group_kernel(int64_t n, const float* __restrict__ times, double split,
                                const DsSlot* __restrict__ slots,
                                const uint32_t* __restrict__ pt_slot, uint32_t* gfirst,
                                uint32_t* __restrict__ pt_group) {
  DS_LOOP(i, n) {
    const uint32_t s = pt_slot[i];
    if (s == kNone) {
      pt_group[i] = kNone;
      continue;
    }
    uint32_t sub = 0u;
    if (times && split > 0.0) {
      const double t0 = (double)times[slots[s].first];
      sub = fabs((double)times[i] - t0) > split ? 1u : 0u;
    }
    const uint32_t g = 2u * s + sub;
    atomicMin(&gfirst[g], (uint32_t)i);
    pt_group[i] = g;
  }
}

__global__ void ds_flags_kernel(int64_t n, const uint32_t* __restrict__ pt_group,
                                const uint32_t* __restrict__ gfirst, uint32_t* __restrict__ flag) {
  DS_LOOP(i, n) {
    const uint32_t g = pt_group[i];
    flag[i] = (g != kNone && gfirst[g] == (uint32_t)i) ? 1u : 0u;
  }
}

__global__ void ds_assign_kernel(int64_t n, const uint32_t* __restrict__ flag,
                                 const uint32_t* __restrict__ prefix,
                                 const uint32_t* __restrict__ pt_group, uint32_t* __restrict__ gmap) {
  DS_LOOP(i, n) {
    if (flag[i]) gmap[pt_group[i]] = prefix[i];
  }
}

__global__ void ds_count_kernel(int64_t n, const uint32_t* __restrict__ pt_group,
                                const uint32_t* __restrict__ gmap, uint32_t* gcount,
                                uint32_t* __restrict__ pt_out) {
  DS_LOOP(i, n) {
    const uint32_t g = pt_group[i];
    if (g == kNone) {
      pt_out[i] = kNone;
      continue;
    }
    const uint32_t v = gmap[g];
    atomicAdd(gcount + v, 1u);
    pt_out[i] = v;
  }
}

__global__ void ds_scatter_kernel(int64_t n, const uint32_t* __restrict__ pt_out,
                                  const uint32_t* __restrict__ goff, uint32_t* gfill,
                                  uint32_t* __restrict__ list) {
  DS_LOOP(i, n) {
    const uint32_t v = pt_out[i];
    if (v == kNone) continue;
    list[goff[v] + atomicAdd(gfill + v, 1u)] = (uint32_t)i;
  }
}

__global__ void ds_finalize_kernel(int64_t n_max, const uint32_t* __restrict__ n_out,
                                   const float* __restrict__ pts, const float* __restrict__ times,
                                   const uint32_t* __restrict__ gcount,
                                   const uint32_t* __restrict__ goff, uint32_t* __restrict__ list,
                                   float* __restrict__ out_pts, float* __restrict__ out_times,
                                   int32_t* __restrict__ out_counts) {
  const int64_t V = min((int64_t)*n_out, n_max);
  DS_LOOP(v, V) {
    const uint32_t c = gcount[v];
    uint32_t* L = list + goff[v];
    for (uint32_t a = 1; a < c; ++a) {  // ascending point index
      const uint32_t x = L[a];
      int b = (int)a - 1;
      while (b >= 0 && L[b] > x) {
        L[b + 1] = L[b];
        --b;
      }
      L[b + 1] = x;
    }
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    bool exact = true;
    for (uint32_t a = 0; a < c; ++a) {
      const int64_t j = L[a];
      df_add(hi[0], lo[0], pts[3 * j], exact);
      df_add(hi[1], lo[1], pts[3 * j + 1], exact);
      df_add(hi[2], lo[2], pts[3 * j + 2], exact);
      if (times) df_add(hi[3], lo[3], times[j], exact);
    }
    double s[4];
    if (exact) {
      for (int k = 0; k < 4; ++k) s[k] = __dadd_rn((double)hi[k], (double)lo[k]);
    } else {
      for (int k = 0; k < 4; ++k) s[k] = 0.0;
      for (uint32_t a = 0; a < c; ++a) {
        const int64_t j = L[a];
        for (int k = 0; k < 3; ++k) s[k] = __dadd_rn(s[k], (double)pts[3 * j + k]);
        if (times) s[3] = __dadd_rn(s[3], (double)times[j]);
      }
    }
    const double N = (double)c, y = __drcp_rn(N);
    for (int k = 0; k < 3; ++k) out_pts[3 * v + k] = __double2float_rn(div_rn(s[k], N, y));
    if (out_times) out_times[v] = __double2float_rn(div_rn(s[3], N, y));
    if (out_counts) out_counts[v] = (int32_t)c;
  }
}

__global__ void ds_offsets_kernel(int32_t n_clouds, int64_t n, const int64_t* __restrict__ off,
                                  const uint32_t* __restrict__ prefix,
                                  const uint32_t* __restrict__ n_out, uint32_t* __restrict__ oo) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > n_clouds) return;
  const int64_t o = off[c];
  oo[c] = o < n ? prefix[o] : *n_out;
}

int grid_of(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 0x7FFFFFFF));
}

}  // namespace
}  // namespace vgicp

extern "C" {

int vgicp_downsample(const float* points, const float* times, const int64_t* offsets,
                     int32_t n_clouds, double resolution, double split, float* out_points,
                     float* out_times, int32_t* out_counts, int64_t* out_offsets,
                     vgicp_stream_t stream) {
  using namespace vgicp;
  if (!(resolution > 0.0) || !std::isfinite(resolution))
    return set_error(VGICP_ERR_INVALID_ARG, "resolution must be positive and finite");
  if (n_clouds <= 0 || !offsets || !out_offsets)
    return set_error(VGICP_ERR_INVALID_ARG, "n_clouds >= 1, offsets and out_offsets required");
  if (offsets[0] != 0) return set_error(VGICP_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (int32_t c = 0; c < n_clouds; ++c)
    if (offsets[c + 1] < offsets[c])
      return set_error(VGICP_ERR_INVALID_ARG, "offsets must be non-decreasing");
  if (!std::isfinite(split)) return set_error(VGICP_ERR_INVALID_ARG, "split must be finite");
  const int64_t n = offsets[n_clouds];
  if (n >= (int64_t)0xFFFFFFFFll) return set_error(VGICP_ERR_INVALID_ARG, "more than 2^32-1 points");
  if (n == 0) {
    for (int32_t c = 0; c <= n_clouds; ++c) out_offsets[c] = 0;
    return VGICP_OK;
  }
  if (!points || !out_points) return set_error(VGICP_ERR_INVALID_ARG, "null points");
  std::vector<int64_t> base((size_t)n_clouds);
  std::vector<uint32_t> mask((size_t)n_clouds);
  int64_t cap = 0;
  for (int32_t c = 0; c < n_clouds; ++c) {
    uint64_t k = 16;
    while (k < 2ull * (uint64_t)std::max<int64_t>(offsets[c + 1] - offsets[c], 1)) k <<= 1;
    base[(size_t)c] = cap;
    mask[(size_t)c] = (uint32_t)(k - 1);
    cap += (int64_t)k;
  }
  if (2 * cap >= (int64_t)0xFFFFFFFFll)
    return set_error(VGICP_ERR_INVALID_ARG, "more than 2^31-1 table slots");
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
    return o;
  };
  const size_t o_off = take(sizeof(int64_t) * (n_clouds + 1));
  const size_t o_base = take(sizeof(int64_t) * n_clouds);
  const size_t o_mask = take(sizeof(uint32_t) * n_clouds);
  const size_t o_status = take(sizeof(int32_t));
  const size_t o_nout = take(sizeof(uint32_t));
  const size_t o_oo = take(sizeof(uint32_t) * (n_clouds + 1));
  const size_t o_slots = take(sizeof(DsSlot) * cap);
  const size_t o_gfirst = take(sizeof(uint32_t) * 2 * cap);
  const size_t o_gmap = take(sizeof(uint32_t) * 2 * cap);
  const size_t o_ptslot = take(sizeof(uint32_t) * n);
  const size_t o_ptgroup = take(sizeof(uint32_t) * n);
  const size_t o_flag = take(sizeof(uint32_t) * n);
  const size_t o_prefix = take(sizeof(uint32_t) * n);
  const size_t o_gcount = take(sizeof(uint32_t) * n);
  const size_t o_goff = take(sizeof(uint32_t) * n);
  const size_t o_list = take(sizeof(uint32_t) * n);
  const size_t o_scan = take(sizeof(uint32_t) * scan_tmp_elems(n));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* d = nullptr;
  VGICP_CUDA_TRY(device_malloc(reinterpret_cast<void**>(&d), off, st, true));
  auto U = [&](size_t o) { return reinterpret_cast<uint32_t*>(d + o); };
  int64_t* d_off = reinterpret_cast<int64_t*>(d + o_off);
  int64_t* d_base = reinterpret_cast<int64_t*>(d + o_base);
  int32_t* d_status = reinterpret_cast<int32_t*>(d + o_status);
  DsSlot* d_slots = reinterpret_cast<DsSlot*>(d + o_slots);
  int rc = VGICP_OK;
  cudaError_t e = cudaMemcpyAsync(d_off, offsets, sizeof(int64_t) * (n_clouds + 1),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * n_clouds, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(U(o_mask), mask.data(), sizeof(uint32_t) * n_clouds,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(U(o_gcount), 0, sizeof(uint32_t) * n, st);
  if (e != cudaSuccess) rc = check_cuda(e, "downsample setup");
  const float inv_r = (float)(1.0 / resolution);
  const int g = grid_of(n), gc = grid_of(cap);
  if (rc == VGICP_OK) {
    ds_init_kernel<<<gc, kThreads, 0, st>>>(d_slots, cap, U(o_gfirst));
    ds_insert_kernel<<<g, kThreads, 0, st>>>(points, n, d_off, n_clouds, inv_r, resolution,
                                             d_base, U(o_mask), d_slots, U(o_ptslot), d_status);
    ds_group_kernel<<<g, kThreads, 0, st>>>(n, times, split, d_slots, U(o_ptslot), U(o_gfirst),
                                            U(o_ptgroup));
    ds_flags_kernel<<<g, kThreads, 0, st>>>(n, U(o_ptgroup), U(o_gfirst), U(o_flag));
    count_launches(4);
    rc = launch_exclusive_scan(U(o_flag), U(o_prefix), n, nullptr, U(o_scan), U(o_nout), st);
  }
  if (rc == VGICP_OK) {
    ds_assign_kernel<<<g, kThreads, 0, st>>>(n, U(o_flag), U(o_prefix), U(o_ptgroup), U(o_gmap));
    // pt_slot is free now: the output voxel of each point
    ds_count_kernel<<<g, kThreads, 0, st>>>(n, U(o_ptgroup), U(o_gmap), U(o_gcount), U(o_ptslot));
    count_launches(2);
    rc = launch_exclusive_scan(U(o_gcount), U(o_goff), n, U(o_nout), U(o_scan), nullptr, st);
  }
  if (rc == VGICP_OK) {
    e = cudaMemsetAsync(U(o_flag), 0, sizeof(uint32_t) * n, st);  // the fill counters
    if (e != cudaSuccess) rc = check_cuda(e, "cudaMemsetAsync");
  }
  if (rc == VGICP_OK) {
    ds_scatter_kernel<<<g, kThreads, 0, st>>>(n, U(o_ptslot), U(o_goff), U(o_flag), U(o_list));
    ds_finalize_kernel<<<g, kThreads, 0, st>>>(n, U(o_nout), points, times, U(o_gcount),
                                               U(o_goff), U(o_list), out_points, out_times,
                                               out_counts);
    ds_offsets_kernel<<<(n_clouds + 1 + 127) / 128, 128, 0, st>>>(n_clouds, n, d_off, U(o_prefix),
                                                                   U(o_nout), U(o_oo));
    count_launches(3);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = check_cuda(e, "downsample kernels");
  }
  std::vector<uint32_t> oo((size_t)n_clouds + 1, 0u);
  int32_t status = 0;
  if (rc == VGICP_OK) {
    e = cudaMemcpyAsync(oo.data(), U(o_oo), sizeof(uint32_t) * oo.size(), cudaMemcpyDeviceToHost,
                        st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = check_cuda(e, "downsample results");
  }
  e = cudaFreeAsync(d, st);
  if (rc == VGICP_OK && e != cudaSuccess) rc = check_cuda(e, "cudaFreeAsync");
  if (rc == VGICP_OK && status == VGICP_ERR_KEY_RANGE)
    return set_error(status, "a point's voxel key is outside [-2^20, 2^20)");
  if (rc == VGICP_OK && status == VGICP_ERR_HASH_FULL)
    return set_error(status, "voxel table probe limit exceeded");
  if (rc == VGICP_OK)
    for (int32_t c = 0; c <= n_clouds; ++c) out_offsets[c] = oo[(size_t)c];
  return rc;
}

}  // extern "C"
