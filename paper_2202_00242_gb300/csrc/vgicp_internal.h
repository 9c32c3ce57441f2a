// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "vgicp.h"
#include "vgicp_device.cuh"

namespace vgicp {

// Device indices the library keeps per-device state for (0 .. kMaxDevices-1).
constexpr int kMaxDevices = 64;

// ---- error reporting -------------------------------------------------------
int set_error(int code, const std::string& msg);
int check_cuda(cudaError_t e, const char* what);  // cudaErrorMemoryAllocation -> OOM
// Every device allocation of the library (cudaMalloc, or cudaMallocAsync on st
// when stream_ordered); fails without allocating while the test hook asks.
cudaError_t device_malloc(void** p, size_t bytes, cudaStream_t st, bool stream_ordered);
#define VGICP_CUDA_TRY(call)                                   \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return check_cuda(e__, #call);     \
  } while (0)

// ---- map storage -----------------------------------------------------------
// One build batch: n_maps maps built from concatenated clouds.  All device
// buffers are sized at creation so that rebuilds allocate nothing.
struct MapSet {
  int refcount = 0;
  int device = 0;
  int32_t n_maps = 0;
  double resolution = 0.0;
  int32_t max_probe = 64;
  int64_t n_total = 0;    // points over all maps
  int64_t cap_total = 0;  // slots over all maps
  std::vector<int64_t> point_off;  // n_maps + 1
  std::vector<int64_t> slot_base;  // n_maps
  std::vector<uint32_t> cap;       // n_maps
  std::vector<int64_t> vslot_base; // n_maps + 1: lookup-table regions, sized from the voxel
  int64_t vcap_total = 0;          //   counts of the first build (empty before it)
  // device: per-map metadata
  int64_t* d_point_off = nullptr;  // n_maps + 1
  int64_t* d_slot_base = nullptr;  // n_maps
  int64_t* d_vslot_base = nullptr; // n_maps + 1
  uint32_t* d_cap_mask = nullptr;  // n_maps
  uint32_t* d_vbase = nullptr;     // n_maps + 1: first global voxel index of each map
  // device: the maps
  Slot* d_slots = nullptr;                  // cap_total (build table)
  VSlot* d_vslots = nullptr;                // vcap_total (lookup tables, inline records),
                                            // in d_vblock
  uint32_t* d_vmask = nullptr;              // n_maps: lookup-table capacity - 1
  float4* d_recs = nullptr;                 // n_total * 3 (V <= n_total)
  unsigned long long* d_vkeys = nullptr;    // n_total (packed keys by voxel)
  int32_t* d_status = nullptr;              // 1
  // device: build scratch (kept for rebuilds)
  uint32_t* d_pt_slot = nullptr;  // n_total: build-table slot of each point
  uint32_t* d_flag = nullptr;     // n_total: voxel id of each point (read at map starts)
  uint32_t* d_vcount = nullptr;   // n_total: points per voxel
  uint32_t* d_voff = nullptr;     // n_total: voxel at each rank
  uint32_t* d_vfill = nullptr;    // n_total: first-point flags, counts by rank, list fill
  uint32_t* d_plist = nullptr;    // n_total: point lists of the voxels, in rank order
  // kept from one build to the next: the lookup-table slot each voxel occupies,
  // so a rebuild empties just those (every other slot is empty already)
  uint32_t* d_lslot_of = nullptr; // n_total: lookup-table slot of each voxel (or kNoSlot)
  bool built = false;             // a build has run: the lookup tables hold only its
                                  // voxels and the build table is empty
  float* d_gpts = nullptr;        // n_total x 3: the clouds grouped by voxel, voxels in
  float* d_gcovs = nullptr;       // n_total x 6   Morton order (within chunks of a map)
  uint32_t* d_goff = nullptr;     // n_total: grouped offset of each Morton rank
  int2* d_chunks = nullptr;       // (map, chunk) pairs for the Morton sort
  int32_t n_chunks = 0;
  uint32_t* d_scan_tmp = nullptr; // scan block sums
  uint32_t* d_num_voxels = nullptr;  // 1 (total V)
  uint32_t* d_num_valid = nullptr;   // 1 (points placed in a voxel)
  size_t scan_tmp_elems = 0;
  void* d_block = nullptr;        // single allocation holding everything above but d_vslots
  void* d_vblock = nullptr;       // the lookup tables (allocated by the first build)
};

// Frees a map set's device memory and the set.
void free_set(MapSet* s);

}  // namespace vgicp

struct vgicp_map {
  vgicp::MapSet* set;
  int32_t index;
};

namespace vgicp {

// ---- kernels (vgicp_build.cu) ---------------------------------------------
int launch_build(MapSet* s, const float* points, const float* covs, cudaStream_t st);

// exclusive scan of n_max uint32 (elements at or beyond *n_dev, if given, count
// as 0); writes the total to *total_dev if non-null.
int launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n_max,
                          const uint32_t* n_dev, uint32_t* block_tmp, uint32_t* total_dev,
                          cudaStream_t st);
size_t scan_tmp_elems(int64_t n_max);

// ---- kernels (vgicp_linearize.cu) ----------------------------------------
struct LinLaunch {
  const WorkItem* items;     // null: uniform items of pair 0 (single factor)
  int32_t n_items;
  int32_t item_size;         // uniform-item mode: points per item
  const PairDesc* pairs;     // null: use `single`
  const MapDesc* maps;       // null: use `single_map`
  const SrcDesc* srcs;       // null: use `single_src`
  PairDesc single;
  MapDesc single_map;
  SrcDesc single_src;
  double* partials;          // n_items x kPartialStride
  int32_t* status;           // device int[2]: [0] nonzero after an internal wait timeout;
                             // [1] work-item counter of the dynamically scheduled kernels
                             //     (both zeroed before every launch)
  int32_t* corr_out;
  int32_t* qkey_out;
  int32_t neighbours;
  int32_t mode;              // 0 linearize (H, b, err); 1 err; 2 gradient; 3 exact gradient
  int32_t variant;           // 1-neighbour kernel: 1 per-point, 2 staged (0 = default)
  int32_t grid;              // 0 = automatic
  cudaEvent_t ev_start;      // optional, recorded around the kernel
  cudaEvent_t ev_stop;
  int64_t wait_limit_ns;     // staged kernel: bound of its mbarrier waits (0 = 2 s)
  int32_t test_withhold_tile;  // staged kernel, tests only: 1 + the tile index each
                               // producer withholds (0 = none)
};
int launch_linearize(const LinLaunch& L, cudaStream_t st);

// Arms the one-shot wait test of the next staged-kernel launch
// (vgicp_test_expire_waits).
int arm_wait_test(int32_t tile, int64_t limit_ns);

// Points per work item and the persistent grid the linearize kernel uses.
int default_item_size();
int linearize_grid(int neighbours, int variant);
int default_variant();

// Sum each pair's partials over its items [span[p].x, span[p].y) in order and
// expand to the 43-double result; span == nullptr means one pair over all
// n_items_single items.  A nonzero *status turns every output into NaN.
// Gradient modes: jr (n_pairs x 36, device, or null) gives J_r^T g instead of g,
// gscale (n_pairs, device, or null) scales the gradient.
int launch_reduce(const double* partials, const int2* span, int32_t n_items_single,
                  int64_t n_pairs, const int32_t* status, double* out, int64_t* inliers,
                  cudaStream_t st, int32_t mode = 0, const double* jr = nullptr,
                  const double* gscale = nullptr);

int device_sm_count();

// Shared host helpers (vgicp_api.cu).
bool finite_pose(const double* T);  // finite rigid transform, last row 0 0 0 1
PairDesc make_pair_desc(const double* T, int32_t map, int32_t src);
MapDesc make_map_desc(const vgicp_map* m);
int check_cloud(const float* pts, const float* covs, int64_t n, const char* what);

// Count of kernels launched by the library (vgicp_launch_count).
void count_launches(int n);

}  // namespace vgicp
