// Host runtime and C ABI of the VGICP library: map handles and their storage,
// argument checking, pose conversion, the batched work planner, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "vgicp.h"
#include "vgicp_internal.h"
#include "vgicp_se3.cuh"

namespace vgicp {

namespace {
thread_local std::string g_error;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint32_t next_pow2(uint64_t x) {
  uint64_t p = 16;
  while (p < x) p <<= 1;
  return (uint32_t)p;
}

}  // namespace

bool finite_pose(const double* T) { return se3::rigid(T); }

PairDesc make_pair_desc(const double* T, int32_t map, int32_t src) {
  return se3::pair_desc(T, map, src);
}

MapDesc make_map_desc(const vgicp_map* m) {
  const MapSet* s = m->set;
  MapDesc d;
  std::memset(&d, 0, sizeof(d));
  d.vslots = s->d_vslots + s->vslot_base[m->index];
  d.vmask = s->d_vmask + m->index;
  d.max_probe = s->max_probe;
  d.inv_r = (float)(1.0 / s->resolution);
  d.margin_scale = d.inv_r * 4.76837158203125e-7f;  // 2^-21
  d.r = s->resolution;
  d.vbase = s->d_vbase + m->index;
  return d;
}

int check_cloud(const float* pts, const float* covs, int64_t n, const char* what) {
  if (n < 0) return set_error(VGICP_ERR_INVALID_ARG, std::string(what) + ": negative size");
  if (n > INT32_MAX)
    return set_error(VGICP_ERR_INVALID_ARG, std::string(what) + ": more than 2^31-1 points");
  if (n > 0 && (!pts || !covs))
    return set_error(VGICP_ERR_INVALID_ARG, std::string(what) + ": null pointer");
  if (((uintptr_t)pts & 3u) || ((uintptr_t)covs & 7u))
    return set_error(VGICP_ERR_INVALID_ARG,
                     std::string(what) + ": points must be 4-byte and covs 8-byte aligned");
  return VGICP_OK;
}

namespace {

int create_set(const int64_t* offsets, int32_t n_maps, double resolution,
               const vgicp_map_opts* opts, cudaStream_t st, MapSet** out) {
  if (!(resolution > 0.0) || !std::isfinite(resolution))
    return set_error(VGICP_ERR_INVALID_ARG, "resolution must be positive and finite");
  if (n_maps <= 0 || !offsets) return set_error(VGICP_ERR_INVALID_ARG, "n_maps must be >= 1");
  if (n_maps > 65535) return set_error(VGICP_ERR_INVALID_ARG, "at most 65535 maps per batch");
  if (offsets[0] != 0) return set_error(VGICP_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (int32_t m = 0; m < n_maps; ++m)
    if (offsets[m + 1] < offsets[m])
      return set_error(VGICP_ERR_INVALID_ARG, "offsets must be non-decreasing");
  int32_t max_probe = opts && opts->max_probe > 0 ? opts->max_probe : 64;
  int32_t cf = opts && opts->capacity_factor > 0 ? opts->capacity_factor : 2;
  if (cf > 64) return set_error(VGICP_ERR_INVALID_ARG, "capacity_factor too large");

  MapSet* s = new MapSet();
  s->n_maps = n_maps;
  s->resolution = resolution;
  s->max_probe = max_probe;
  s->point_off.assign(offsets, offsets + n_maps + 1);
  s->n_total = offsets[n_maps];
  s->slot_base.resize(n_maps);
  s->cap.resize(n_maps);
  int64_t cap_total = 0;
  for (int32_t m = 0; m < n_maps; ++m) {
    int64_t n = offsets[m + 1] - offsets[m];
    uint32_t c = next_pow2((uint64_t)std::max<int64_t>(n, 1) * (uint64_t)cf);
    s->cap[m] = c;
    s->slot_base[m] = cap_total;
    cap_total += c;
  }
  s->cap_total = cap_total;
  if (s->n_total >= (int64_t)0xFFFFFFFFll || cap_total >= (int64_t)0xFFFFFFFFll) {
    delete s;
    return set_error(VGICP_ERR_INVALID_ARG, "more than 2^32-1 points or slots in one batch");
  }
  const int64_t n = s->n_total;
  s->scan_tmp_elems = scan_tmp_elems(std::max<int64_t>(n, 1));
  // one allocation, 256-B aligned sub-buffers
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  const size_t o_point_off = take(sizeof(int64_t) * (n_maps + 1));
  const size_t o_slot_base = take(sizeof(int64_t) * n_maps);
  const size_t o_vslot_base = take(sizeof(int64_t) * (n_maps + 1));
  const size_t o_cap_mask = take(sizeof(uint32_t) * n_maps);
  const size_t o_vbase = take(sizeof(uint32_t) * (n_maps + 1));
  const size_t o_slots = take(sizeof(Slot) * cap_total);
  const size_t o_vmask = take(sizeof(uint32_t) * n_maps);
  const size_t o_recs = take(sizeof(float4) * kRecordF4 * n);
  const size_t o_vkeys = take(sizeof(unsigned long long) * n);
  const size_t o_status = take(sizeof(int32_t));
  const size_t o_num_vox = take(sizeof(uint32_t));
  const size_t o_num_valid = take(sizeof(uint32_t));
  const size_t o_pt_slot = take(sizeof(uint32_t) * n);
  const size_t o_flag = take(sizeof(uint32_t) * n);
  const size_t o_vcount = take(sizeof(uint32_t) * n);
  const size_t o_voff = take(sizeof(uint32_t) * n);
  const size_t o_vfill = take(sizeof(uint32_t) * n);
  const size_t o_plist = take(sizeof(uint32_t) * n);
  const size_t o_lslot_of = take(sizeof(uint32_t) * n);
  std::vector<int2> chunks;
  for (int32_t m = 0; m < n_maps; ++m) {
    const int64_t nm = offsets[m + 1] - offsets[m];
    for (int64_t c = 0; c * kMortonChunk < std::max<int64_t>(nm, 1); ++c)
      chunks.push_back(make_int2(m, (int)c));
  }
  s->n_chunks = (int32_t)chunks.size();
  const size_t o_chunks = take(sizeof(int2) * chunks.size());
  const size_t o_goff = take(sizeof(uint32_t) * n);
  const size_t o_gpts = take(sizeof(float) * 3 * n);
  const size_t o_gcovs = take(sizeof(float) * 6 * n);
  const size_t o_scan = take(sizeof(uint32_t) * s->scan_tmp_elems);
  cudaError_t e = device_malloc(&s->d_block, off, nullptr, false);
  if (e != cudaSuccess) {
    delete s;
    cudaGetLastError();
    return set_error(VGICP_ERR_OOM, std::string("voxel map allocation of ") +
                                        std::to_string(off) + " bytes failed");
  }
  char* b = static_cast<char*>(s->d_block);
  s->d_point_off = reinterpret_cast<int64_t*>(b + o_point_off);
  s->d_slot_base = reinterpret_cast<int64_t*>(b + o_slot_base);
  s->d_vslot_base = reinterpret_cast<int64_t*>(b + o_vslot_base);
  s->d_cap_mask = reinterpret_cast<uint32_t*>(b + o_cap_mask);
  s->d_vbase = reinterpret_cast<uint32_t*>(b + o_vbase);
  s->d_slots = reinterpret_cast<Slot*>(b + o_slots);
  s->d_vmask = reinterpret_cast<uint32_t*>(b + o_vmask);
  s->d_recs = reinterpret_cast<float4*>(b + o_recs);
  s->d_vkeys = reinterpret_cast<unsigned long long*>(b + o_vkeys);
  s->d_status = reinterpret_cast<int32_t*>(b + o_status);
  s->d_num_voxels = reinterpret_cast<uint32_t*>(b + o_num_vox);
  s->d_num_valid = reinterpret_cast<uint32_t*>(b + o_num_valid);
  s->d_pt_slot = reinterpret_cast<uint32_t*>(b + o_pt_slot);
  s->d_flag = reinterpret_cast<uint32_t*>(b + o_flag);
  s->d_vcount = reinterpret_cast<uint32_t*>(b + o_vcount);
  s->d_voff = reinterpret_cast<uint32_t*>(b + o_voff);
  s->d_vfill = reinterpret_cast<uint32_t*>(b + o_vfill);
  s->d_plist = reinterpret_cast<uint32_t*>(b + o_plist);
  s->d_lslot_of = reinterpret_cast<uint32_t*>(b + o_lslot_of);
  s->d_gpts = reinterpret_cast<float*>(b + o_gpts);
  s->d_goff = reinterpret_cast<uint32_t*>(b + o_goff);
  s->d_chunks = reinterpret_cast<int2*>(b + o_chunks);
  s->d_gcovs = reinterpret_cast<float*>(b + o_gcovs);
  s->d_scan_tmp = reinterpret_cast<uint32_t*>(b + o_scan);
  cudaGetDevice(&s->device);
  std::vector<uint32_t> mask(n_maps);
  for (int32_t m = 0; m < n_maps; ++m) mask[m] = s->cap[m] - 1u;
  // metadata is small: synchronous copies keep the host vectors' lifetime simple
  e = cudaMemcpy(s->d_point_off, s->point_off.data(), sizeof(int64_t) * (n_maps + 1),
                 cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_slot_base, s->slot_base.data(), sizeof(int64_t) * n_maps,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_cap_mask, mask.data(), sizeof(uint32_t) * n_maps, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_chunks, chunks.data(), sizeof(int2) * chunks.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_set(s);
    return check_cuda(e, "cudaMemcpy(map metadata)");
  }
  (void)st;
  *out = s;
  return VGICP_OK;
}

void release_set(MapSet* s) {
  if (--s->refcount == 0) free_set(s);
}

int sm_count_cache[kMaxDevices] = {0};
std::mutex sm_mutex;
std::atomic<int64_t> g_launches{0};

}  // namespace

void free_set(MapSet* s) {
  cudaFree(s->d_vblock);
  cudaFree(s->d_block);
  delete s;
}

int set_error(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  g_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // not sticky: clear it so the context stays usable
    return VGICP_ERR_OOM;
  }
  return VGICP_ERR_CUDA;
}

// Allocations the test hook makes fail (vgicp_test_fail_allocations).
std::atomic<int32_t> g_fail_allocs{0};

cudaError_t device_malloc(void** p, size_t bytes, cudaStream_t st, bool stream_ordered) {
  int32_t k = g_fail_allocs.load(std::memory_order_relaxed);
  while (k > 0) {
    if (g_fail_allocs.compare_exchange_weak(k, k - 1)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return stream_ordered ? cudaMallocAsync(p, bytes, st) : cudaMalloc(p, bytes);
}

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int device_sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices) dev = 0;
  std::lock_guard<std::mutex> g(sm_mutex);
  if (sm_count_cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
    sm_count_cache[dev] = n;
  }
  return sm_count_cache[dev];
}

}  // namespace vgicp

using namespace vgicp;

extern "C" {

const char* vgicp_last_error_string(void) { return g_error.c_str(); }

int vgicp_version(void) { return 10000; }

int64_t vgicp_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int vgicp_test_fail_allocations(int32_t count) {
  if (count < 0) return set_error(VGICP_ERR_INVALID_ARG, "negative count");
  g_fail_allocs.store(count, std::memory_order_relaxed);
  return VGICP_OK;
}

int vgicp_test_expire_waits(int32_t tile, int64_t limit_ns) {
  g_error.clear();
  return arm_wait_test(tile, limit_ns);
}

int vgicp_build_voxelmaps(const float* points, const float* covs, const int64_t* offsets,
                          int32_t n_maps, double resolution, const vgicp_map_opts* opts,
                          vgicp_stream_t stream, vgicp_map** out) {
  g_error.clear();
  if (!out) return set_error(VGICP_ERR_INVALID_ARG, "out is null");
  if (n_maps <= 0 || !offsets) return set_error(VGICP_ERR_INVALID_ARG, "n_maps must be >= 1");
  int rc = check_cloud(points, covs, offsets[n_maps], "target clouds");
  if (rc) return rc;
  MapSet* s = nullptr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  rc = create_set(offsets, n_maps, resolution, opts, st, &s);
  if (rc) return rc;
  rc = launch_build(s, points, covs, st);
  if (rc) {
    free_set(s);
    return rc;
  }
  for (int32_t m = 0; m < n_maps; ++m) {
    out[m] = new vgicp_map{s, m};
    ++s->refcount;
  }
  return VGICP_OK;
}

int vgicp_build_voxelmap(const float* points, const float* covs, int64_t n, double resolution,
                         const vgicp_map_opts* opts, vgicp_stream_t stream, vgicp_map** out) {
  if (n < 0) return set_error(VGICP_ERR_INVALID_ARG, "negative size");
  const int64_t off[2] = {0, n};
  return vgicp_build_voxelmaps(points, covs, off, 1, resolution, opts, stream, out);
}

int vgicp_rebuild_voxelmaps(vgicp_map* const* maps, int32_t n_maps, const float* points,
                            const float* covs, vgicp_stream_t stream) {
  g_error.clear();
  if (!maps || n_maps <= 0 || !maps[0]) return set_error(VGICP_ERR_INVALID_ARG, "no maps");
  MapSet* s = maps[0]->set;
  if (n_maps != s->n_maps)
    return set_error(VGICP_ERR_INVALID_ARG, "rebuild needs every map of the batch");
  for (int32_t m = 0; m < n_maps; ++m)
    if (!maps[m] || maps[m]->set != s || maps[m]->index != m)
      return set_error(VGICP_ERR_INVALID_ARG, "maps are not one batch in creation order");
  int rc = check_cloud(points, covs, s->n_total, "target clouds");
  if (rc) return rc;
  return launch_build(s, points, covs, reinterpret_cast<cudaStream_t>(stream));
}

int vgicp_destroy_voxelmap(vgicp_map* map) {
  g_error.clear();
  if (!map) return VGICP_OK;
  release_set(map->set);
  delete map;
  return VGICP_OK;
}

int vgicp_voxelmap_status(const vgicp_map* map, vgicp_stream_t stream) {
  g_error.clear();
  if (!map) return set_error(VGICP_ERR_INVALID_ARG, "map is null");
  VGICP_CUDA_TRY(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  int32_t st = 0;
  VGICP_CUDA_TRY(cudaMemcpy(&st, map->set->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st == VGICP_ERR_HASH_FULL)
    return set_error(st, "voxel map build: a voxel did not fit within max_probe slots");
  if (st == VGICP_ERR_KEY_RANGE)
    return set_error(st, "voxel map build: a point's voxel key is outside [-2^20, 2^20) "
                         "(coordinate too large for the resolution, or not finite)");
  return st;
}

int vgicp_voxelmap_info(const vgicp_map* map, vgicp_stream_t stream, int64_t* num_voxels,
                        int64_t* capacity) {
  g_error.clear();
  if (!map) return set_error(VGICP_ERR_INVALID_ARG, "map is null");
  VGICP_CUDA_TRY(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  uint32_t vb[2];
  VGICP_CUDA_TRY(cudaMemcpy(vb, map->set->d_vbase + map->index, sizeof(vb),
                            cudaMemcpyDeviceToHost));
  if (num_voxels) *num_voxels = (int64_t)vb[1] - (int64_t)vb[0];
  if (capacity) *capacity = map->set->cap[map->index];
  return VGICP_OK;
}

int vgicp_voxelmap_grouped_cloud(const vgicp_map* map, vgicp_stream_t stream, float* points,
                                 float* covs) {
  g_error.clear();
  if (!map) return set_error(VGICP_ERR_INVALID_ARG, "map is null");
  const MapSet* s = map->set;
  const int64_t a = s->point_off[map->index], b = s->point_off[map->index + 1];
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (b > a && points)
    VGICP_CUDA_TRY(cudaMemcpyAsync(points, s->d_gpts + 3 * a, sizeof(float) * 3 * (b - a),
                                   cudaMemcpyDeviceToDevice, st));
  if (b > a && covs)
    VGICP_CUDA_TRY(cudaMemcpyAsync(covs, s->d_gcovs + 6 * a, sizeof(float) * 6 * (b - a),
                                   cudaMemcpyDeviceToDevice, st));
  return VGICP_OK;
}

int vgicp_voxelmap_export(const vgicp_map* map, vgicp_stream_t stream, int64_t max_voxels,
                          int64_t* keys, int32_t* counts, float* means, float* covs) {
  int64_t V = 0;
  int rc = vgicp_voxelmap_info(map, stream, &V, nullptr);
  if (rc) return rc;
  if (V > max_voxels) return set_error(VGICP_ERR_INVALID_ARG, "max_voxels smaller than V");
  if (V == 0) return VGICP_OK;
  const MapSet* s = map->set;
  uint32_t vb = 0;
  VGICP_CUDA_TRY(cudaMemcpy(&vb, s->d_vbase + map->index, sizeof(vb), cudaMemcpyDeviceToHost));
  std::vector<unsigned long long> k((size_t)V);
  std::vector<float4> r((size_t)V * kRecordF4);
  VGICP_CUDA_TRY(cudaMemcpy(k.data(), s->d_vkeys + vb, sizeof(unsigned long long) * V,
                            cudaMemcpyDeviceToHost));
  VGICP_CUDA_TRY(cudaMemcpy(r.data(), s->d_recs + (size_t)vb * kRecordF4,
                            sizeof(float4) * kRecordF4 * V, cudaMemcpyDeviceToHost));
  const unsigned long long fm = (1ull << kKeyBits) - 1ull;
  for (int64_t v = 0; v < V; ++v) {
    if (keys) {
      keys[3 * v + 0] = (int64_t)((k[v] >> (2 * kKeyBits)) & fm) - kKeyBias;
      keys[3 * v + 1] = (int64_t)((k[v] >> kKeyBits) & fm) - kKeyBias;
      keys[3 * v + 2] = (int64_t)(k[v] & fm) - kKeyBias;
    }
    const float4 a = r[3 * v], b = r[3 * v + 1], c = r[3 * v + 2];
    if (counts) {
      uint32_t cnt;
      std::memcpy(&cnt, &a.w, sizeof(cnt));
      counts[v] = (int32_t)cnt;
    }
    if (means) {
      means[3 * v + 0] = a.x;
      means[3 * v + 1] = a.y;
      means[3 * v + 2] = a.z;
    }
    if (covs) {
      covs[6 * v + 0] = b.x;
      covs[6 * v + 1] = b.y;
      covs[6 * v + 2] = b.z;
      covs[6 * v + 3] = b.w;
      covs[6 * v + 4] = c.x;
      covs[6 * v + 5] = c.y;
    }
  }
  return VGICP_OK;
}

int vgicp_linearize(const vgicp_map* map, const float* src_points, const float* src_covs,
                    int64_t n_src, const double* T_target_source, double* out, int64_t* inliers,
                    const vgicp_lin_opts* opts, vgicp_stream_t stream) {
  g_error.clear();
  if (!map || !out || !inliers || !T_target_source)
    return set_error(VGICP_ERR_INVALID_ARG, "null map, output or pose");
  int rc = check_cloud(src_points, src_covs, n_src, "source cloud");
  if (rc) return rc;
  if (!finite_pose(T_target_source))
    return set_error(VGICP_ERR_INVALID_ARG, "pose must be a finite rigid transform");
  const int neighbours = opts && opts->neighbours ? opts->neighbours : 1;
  if (neighbours != 1 && neighbours != 27)
    return set_error(VGICP_ERR_INVALID_ARG, "neighbours must be 1 or 27");
  if (opts && (opts->variant < 0 || opts->variant > 3))
    return set_error(VGICP_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  int item = opts && opts->tile > 0 ? opts->tile : 0;
  if (item == 0) {
    // spread one factor over the persistent grid, 256..16K points per item
    const int64_t target_items =
        linearize_grid(neighbours, opts && opts->variant ? opts->variant : default_variant());
    int64_t t = (n_src + target_items - 1) / std::max<int64_t>(target_items, 1);
    t = std::max<int64_t>(256, std::min<int64_t>(default_item_size(), (t + 255) / 256 * 256));
    item = (int)t;
  }
  const int32_t n_items = (int32_t)((n_src + item - 1) / item);

  LinLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.items = nullptr;
  L.n_items = n_items;
  L.item_size = item;
  L.single = make_pair_desc(T_target_source, 0, 0);
  L.single_map = make_map_desc(map);
  L.single_src = SrcDesc{src_points, src_covs, n_src};
  L.corr_out = opts ? opts->corr_out : nullptr;
  L.qkey_out = opts ? opts->qkey_out : nullptr;
  L.neighbours = neighbours;
  L.variant = opts ? opts->variant : 0;
  L.grid = opts ? opts->grid : 0;
  L.ev_start = opts ? static_cast<cudaEvent_t>(opts->kernel_start) : nullptr;
  L.ev_stop = opts ? static_cast<cudaEvent_t>(opts->kernel_stop) : nullptr;
  // scratch: partials (n_items x 32 doubles) followed by the status word
  char* scratch = nullptr;
  const size_t part_bytes = sizeof(double) * kPartialStride * std::max<int32_t>(n_items, 1);
  VGICP_CUDA_TRY(device_malloc(reinterpret_cast<void**>(&scratch), part_bytes + 256, st, true));
  L.partials = reinterpret_cast<double*>(scratch);
  L.status = reinterpret_cast<int32_t*>(scratch + part_bytes);
  cudaError_t e = cudaMemsetAsync(L.status, 0, 2 * sizeof(int32_t), st);
  rc = e == cudaSuccess ? VGICP_OK : check_cuda(e, "cudaMemsetAsync");
  if (rc == VGICP_OK) rc = launch_linearize(L, st);
  if (rc == VGICP_OK)
    rc = launch_reduce(L.partials, nullptr, n_items, 1, L.status, out, inliers, st);
  e = cudaFreeAsync(scratch, st);
  if (rc == VGICP_OK && e != cudaSuccess) rc = check_cuda(e, "cudaFreeAsync");
  return rc;
}

static int batched_impl(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                        int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                        const double* poses, double* out, int64_t* inliers,
                        const vgicp_lin_opts* opts, vgicp_stream_t stream, int32_t mode);

int vgicp_linearize_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                            int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                            const double* poses, double* out, int64_t* inliers,
                            const vgicp_lin_opts* opts, vgicp_stream_t stream) {
  return batched_impl(maps, n_maps, sources, n_sources, pairs, n_pairs, poses, out, inliers, opts,
                      stream, 0);
}

int vgicp_evaluate_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                           int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                           const double* poses, int32_t mode, double* out, int64_t* inliers,
                           const vgicp_lin_opts* opts, vgicp_stream_t stream) {
  if (mode < 1 || mode > 3)
    return set_error(VGICP_ERR_INVALID_ARG, "mode must be 1 (cost), 2 (gradient) or 3 (exact)");
  return batched_impl(maps, n_maps, sources, n_sources, pairs, n_pairs, poses, out, inliers, opts,
                      stream, mode);
}

int vgicp_backward_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                           int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                           const double* poses, int32_t exact, double* out, int64_t* inliers,
                           const vgicp_lin_opts* opts, vgicp_stream_t stream) {
  if (exact != 0 && exact != 1) return set_error(VGICP_ERR_INVALID_ARG, "exact must be 0 or 1");
  return batched_impl(maps, n_maps, sources, n_sources, pairs, n_pairs, poses, out, inliers, opts,
                      stream, exact ? 3 : 2);
}

int vgicp_overlap_batched(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                          int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                          const double* poses, int64_t* inliers, const vgicp_lin_opts* opts,
                          vgicp_stream_t stream) {
  if (opts && opts->neighbours != 0 && opts->neighbours != 1)
    return set_error(VGICP_ERR_INVALID_ARG, "the overlap rate uses the 1-neighbour lookup");
  return batched_impl(maps, n_maps, sources, n_sources, pairs, n_pairs, poses, nullptr, inliers,
                      opts, stream, 4);
}

static int batched_impl(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                        int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                        const double* poses, double* out, int64_t* inliers,
                        const vgicp_lin_opts* opts, vgicp_stream_t stream, int32_t mode) {
  g_error.clear();
  if (n_pairs < 0) return set_error(VGICP_ERR_INVALID_ARG, "negative n_pairs");
  if (n_pairs == 0) return VGICP_OK;
  if (!maps || n_maps <= 0 || !sources || n_sources <= 0 || !pairs || !poses ||
      (!out && mode != 4) || !inliers)
    return set_error(VGICP_ERR_INVALID_ARG, "null argument");
  if (n_pairs > INT32_MAX / 2) return set_error(VGICP_ERR_INVALID_ARG, "too many pairs");
  const int neighbours = opts && opts->neighbours ? opts->neighbours : 1;
  if (neighbours != 1 && neighbours != 27)
    return set_error(VGICP_ERR_INVALID_ARG, "neighbours must be 1 or 27");
  if (opts && (opts->corr_out || opts->qkey_out))
    return set_error(VGICP_ERR_INVALID_ARG, "corr_out/qkey_out are single-factor options");
  if (opts && (opts->variant < 0 || opts->variant > 3))
    return set_error(VGICP_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  for (int32_t m = 0; m < n_maps; ++m)
    if (!maps[m]) return set_error(VGICP_ERR_INVALID_ARG, "null map handle");
  // resolve sources: user clouds, or a map's own voxel-grouped cloud
  std::vector<SrcDesc> sd((size_t)n_sources);
  for (int32_t c = 0; c < n_sources; ++c) {
    if (sources[c].map) {
      const vgicp_map* m = sources[c].map;
      const MapSet* ms = m->set;
      const int64_t a = ms->point_off[m->index], b = ms->point_off[m->index + 1];
      sd[(size_t)c] = SrcDesc{ms->d_gpts + 3 * a, ms->d_gcovs + 6 * a, b - a};
    } else {
      int rc = check_cloud(sources[c].points, sources[c].covs, sources[c].n, "source cloud");
      if (rc) return rc;
      sd[(size_t)c] = SrcDesc{sources[c].points, sources[c].covs, sources[c].n};
    }
  }
  const int item = opts && opts->tile > 0 ? opts->tile : default_item_size();
  // host planner: pair descriptors; work items (chunks of each pair's source),
  // emitted in order of (target map, source) so that concurrently running CTAs
  // share a few target maps in L2; span[p] = the items of pair p.
  std::vector<PairDesc> pd((size_t)n_pairs);
  std::vector<int64_t> order((size_t)n_pairs);
  for (int64_t p = 0; p < n_pairs; ++p) {
    const int32_t m = pairs[2 * p], c = pairs[2 * p + 1];
    if (m < 0 || m >= n_maps || c < 0 || c >= n_sources)
      return set_error(VGICP_ERR_INVALID_ARG, "pair index out of range");
    if (!finite_pose(poses + 16 * p))
      return set_error(VGICP_ERR_INVALID_ARG,
                       "pose " + std::to_string(p) + " is not a finite rigid transform");
    pd[(size_t)p] = make_pair_desc(poses + 16 * p, m, c);
    order[(size_t)p] = p;
  }
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return pairs[2 * a] != pairs[2 * b] ? pairs[2 * a] < pairs[2 * b]
                                        : pairs[2 * a + 1] < pairs[2 * b + 1];
  });
  std::vector<int2> span((size_t)n_pairs);
  std::vector<WorkItem> items;
  for (int64_t q = 0; q < n_pairs; ++q) {
    const int64_t p = order[(size_t)q];
    const int64_t n = sd[(size_t)pairs[2 * p + 1]].n;
    const int32_t first = (int32_t)items.size();
    for (int64_t b = 0; b < n; b += item)
      items.push_back(WorkItem{(int32_t)p, (int32_t)b, (int32_t)std::min<int64_t>(n, b + item), 0});
    span[(size_t)p] = make_int2(first, (int32_t)items.size());
    if (items.size() > (size_t)INT32_MAX / 2)
      return set_error(VGICP_ERR_INVALID_ARG, "too many work items");
  }
  const int64_t n_items = (int64_t)items.size();
  std::vector<MapDesc> md((size_t)n_maps);
  for (int32_t m = 0; m < n_maps; ++m) md[(size_t)m] = make_map_desc(maps[m]);

  // one device buffer: descriptors, items, spans | status, partials
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  const size_t o_pd = take(sizeof(PairDesc) * pd.size());
  const size_t o_md = take(sizeof(MapDesc) * md.size());
  const size_t o_sd = take(sizeof(SrcDesc) * sd.size());
  const size_t o_items = take(sizeof(WorkItem) * items.size());
  const size_t o_span = take(sizeof(int2) * span.size());
  const size_t upload = off;
  const size_t o_status = take(sizeof(int32_t));
  const size_t o_part = take(sizeof(double) * kPartialStride * std::max<int64_t>(n_items, 1));
  std::vector<char> host(upload);
  std::memcpy(host.data() + o_pd, pd.data(), sizeof(PairDesc) * pd.size());
  std::memcpy(host.data() + o_md, md.data(), sizeof(MapDesc) * md.size());
  std::memcpy(host.data() + o_sd, sd.data(), sizeof(SrcDesc) * sd.size());
  if (!items.empty())
    std::memcpy(host.data() + o_items, items.data(), sizeof(WorkItem) * items.size());
  std::memcpy(host.data() + o_span, span.data(), sizeof(int2) * span.size());

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* dev = nullptr;
  VGICP_CUDA_TRY(device_malloc(reinterpret_cast<void**>(&dev), off, st, true));
  int rc = VGICP_OK;
  // (a copy from pageable memory returns once the source has been staged, so
  // `host` may be released when this function returns)
  cudaError_t e = cudaMemcpyAsync(dev, host.data(), upload, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = check_cuda(e, "cudaMemcpyAsync(plan)");
  if (rc == VGICP_OK) {
    e = cudaMemsetAsync(dev + o_status, 0, 2 * sizeof(int32_t), st);
    if (e != cudaSuccess) rc = check_cuda(e, "cudaMemsetAsync");
  }
  if (rc == VGICP_OK) {
    LinLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.items = reinterpret_cast<const WorkItem*>(dev + o_items);
    L.n_items = (int32_t)n_items;
    L.item_size = item;
    L.pairs = reinterpret_cast<const PairDesc*>(dev + o_pd);
    L.maps = reinterpret_cast<const MapDesc*>(dev + o_md);
    L.srcs = reinterpret_cast<const SrcDesc*>(dev + o_sd);
    L.partials = reinterpret_cast<double*>(dev + o_part);
    L.status = reinterpret_cast<int32_t*>(dev + o_status);
    L.neighbours = neighbours;
    L.mode = mode;
    L.variant = opts ? opts->variant : 0;
    L.grid = opts ? opts->grid : 0;
    L.ev_start = opts ? static_cast<cudaEvent_t>(opts->kernel_start) : nullptr;
    L.ev_stop = opts ? static_cast<cudaEvent_t>(opts->kernel_stop) : nullptr;
    rc = launch_linearize(L, st);
    if (rc == VGICP_OK)
      rc = launch_reduce(L.partials, reinterpret_cast<const int2*>(dev + o_span), 0, n_pairs,
                         L.status, out, inliers, st, mode);
  }
  e = cudaFreeAsync(dev, st);
  if (rc == VGICP_OK && e != cudaSuccess) rc = check_cuda(e, "cudaFreeAsync");
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Single-factor linearization without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// real-time front-end that sizes its whole GPU footprint at start-up and must
// not take the allocator's locks or latency inside its control loop, or a host
// framework that hands a plugin a stream and forbids allocations on it.  This
// entry point serves them.  It keeps the per-item partial sums and the status
// word in one fixed array in device memory, declared below, so it calls no
// cudaMalloc / cudaFree of any kind.  The array is created when the library is
// loaded and every GPU that loads the library keeps it until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int32_t kNoAllocMaxItems = 4096;  // work items per call (1 MiB of partials)
// partials: kNoAllocMaxItems x kPartialStride doubles, then 32 doubles of which
// the first 4 bytes are the status word
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxItems + 1) * kPartialStride];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The array's name
// in host code only stands for the symbol; the address must be asked for with
// that device current.  Done once per device, on its first call.
int noalloc_scratch(double** out) {
  int dev = 0;
  VGICP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(VGICP_ERR_INVALID_ARG, "device index beyond the supported range");
  std::lock_guard<std::mutex> g(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return VGICP_OK;
}

}  // namespace

extern "C" int vgicp_linearize_noalloc(const vgicp_map* map, const float* src_points,
                                       const float* src_covs, int64_t n_src,
                                       const double* T_target_source, double* out,
                                       int64_t* inliers, const vgicp_lin_opts* opts,
                                       vgicp_stream_t stream) {
  g_error.clear();
  if (!map || !out || !inliers || !T_target_source)
    return set_error(VGICP_ERR_INVALID_ARG, "null map, output or pose");
  int rc = check_cloud(src_points, src_covs, n_src, "source cloud");
  if (rc) return rc;
  if (!finite_pose(T_target_source))
    return set_error(VGICP_ERR_INVALID_ARG, "pose must be a finite rigid transform");
  const int neighbours = opts && opts->neighbours ? opts->neighbours : 1;
  if (neighbours != 1 && neighbours != 27)
    return set_error(VGICP_ERR_INVALID_ARG, "neighbours must be 1 or 27");
  if (opts && (opts->variant < 0 || opts->variant > 3))
    return set_error(VGICP_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  int item = opts && opts->tile > 0 ? opts->tile : 0;
  if (item == 0) {
    const int64_t target_items =
        linearize_grid(neighbours, opts && opts->variant ? opts->variant : default_variant());
    int64_t t = (n_src + target_items - 1) / std::max<int64_t>(target_items, 1);
    t = std::max<int64_t>(256, std::min<int64_t>(default_item_size(), (t + 255) / 256 * 256));
    item = (int)t;
  }
  const int64_t n_items = (n_src + item - 1) / item;
  if (n_items > kNoAllocMaxItems)
    return set_error(VGICP_ERR_INVALID_ARG,
                     "vgicp_linearize_noalloc: " + std::to_string(n_items) +
                         " work items exceed its fixed scratch of " +
                         std::to_string(kNoAllocMaxItems) +
                         " (n_src / item size must be at most that; raise opts->tile or use "
                         "vgicp_linearize)");
  double* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  LinLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.items = nullptr;
  L.n_items = (int32_t)n_items;
  L.item_size = item;
  L.single = make_pair_desc(T_target_source, 0, 0);
  L.single_map = make_map_desc(map);
  L.single_src = SrcDesc{src_points, src_covs, n_src};
  L.corr_out = opts ? opts->corr_out : nullptr;
  L.qkey_out = opts ? opts->qkey_out : nullptr;
  L.neighbours = neighbours;
  L.variant = opts ? opts->variant : 0;
  L.grid = opts ? opts->grid : 0;
  L.ev_start = opts ? static_cast<cudaEvent_t>(opts->kernel_start) : nullptr;
  L.ev_stop = opts ? static_cast<cudaEvent_t>(opts->kernel_stop) : nullptr;
  L.partials = scratch;
  L.status = reinterpret_cast<int32_t*>(scratch + (size_t)kNoAllocMaxItems * kPartialStride);
  // the array keeps the previous call's contents: the status word must start at
  // zero; every partial the reduction reads is written by this call
  VGICP_CUDA_TRY(cudaMemsetAsync(L.status, 0, 2 * sizeof(int32_t), st));
  rc = launch_linearize(L, st);
  if (rc == VGICP_OK)
    rc = launch_reduce(L.partials, nullptr, (int32_t)n_items, 1, L.status, out, inliers, st);
  return rc;
}
