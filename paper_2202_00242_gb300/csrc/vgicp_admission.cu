// Admission scheduling for factor sets whose maps and clouds do not all fit in
// device memory at once (the large-map workload of the global mapping module,
// arXiv 2202.00242 Sec. III-F: the factor count grows with every revisit).
// Host-only.
#include <algorithm>
#include <cstdint>
#include <string>
#include <unordered_set>
#include <vector>

#include "vgicp.h"
#include "vgicp_device.cuh"
#include "vgicp_internal.h"

extern "C" {

int64_t vgicp_voxelmap_bytes(int64_t n_points, const vgicp_map_opts* opts) {
  if (n_points < 0) return -1;
  const int64_t cf = opts && opts->capacity_factor > 0 ? opts->capacity_factor : 2;
  int64_t cap = 16, vcap = 16;
  while (cap < std::max<int64_t>(n_points, 1) * cf) cap <<= 1;
  while (vcap < std::max<int64_t>(n_points, 8) * (int64_t)vgicp::kLookupLoad) vcap <<= 1;
  // build table + lookup table + records + keys + grouped cloud + scratch
  return cap * 16 + vcap * 64 + n_points * (48 + 8 + 36 + 4 * 9) + 4096;
}

int vgicp_admission_schedule(const int64_t* map_bytes, int32_t n_maps, const int64_t* src_bytes,
                             int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                             int64_t budget, int32_t src_is_map, int32_t* batch_of_pair,
                             int32_t* n_batches) {
  using vgicp::set_error;
  if (!map_bytes || !pairs || !batch_of_pair || !n_batches || n_maps <= 0 || n_pairs < 0 ||
      (!src_is_map && (!src_bytes || n_sources <= 0)))
    return set_error(VGICP_ERR_INVALID_ARG, "null or empty schedule argument");
  if (src_is_map) n_sources = n_maps;
  std::vector<int64_t> order((size_t)n_pairs);
  for (int64_t p = 0; p < n_pairs; ++p) {
    const int32_t m = pairs[2 * p], c = pairs[2 * p + 1];
    if (m < 0 || m >= n_maps || c < 0 || c >= n_sources)
      return set_error(VGICP_ERR_INVALID_ARG, "pair index out of range");
    order[(size_t)p] = p;
  }
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return pairs[2 * a] != pairs[2 * b] ? pairs[2 * a] < pairs[2 * b]
                                        : pairs[2 * a + 1] < pairs[2 * b + 1];
  });
  // resident items of the current batch: maps as m, sources as n_maps + c (or m)
  std::unordered_set<int64_t> resident;
  int64_t used = 0;
  int32_t batch = 0;
  auto item_bytes = [&](int64_t id) {
    return id < n_maps ? map_bytes[id] : src_bytes[id - n_maps];
  };
  for (int64_t q = 0; q < n_pairs; ++q) {
    const int64_t p = order[(size_t)q];
    const int64_t need[2] = {pairs[2 * p], src_is_map ? (int64_t)pairs[2 * p + 1]
                                                      : (int64_t)n_maps + pairs[2 * p + 1]};
    int64_t add = 0;
    for (int k = 0; k < 2; ++k)
      if (!resident.count(need[k]) && !(k == 1 && need[1] == need[0])) add += item_bytes(need[k]);
    if (used + add > budget && !resident.empty()) {
      ++batch;
      resident.clear();
      used = 0;
      add = item_bytes(need[0]) + (need[1] == need[0] ? 0 : item_bytes(need[1]));
    }
    if (add > budget)
      return set_error(VGICP_ERR_INVALID_ARG,
                       "pair " + std::to_string(p) + " alone exceeds the admission budget");
    resident.insert(need[0]);
    resident.insert(need[1]);
    used += add;
    batch_of_pair[p] = batch;
  }
  *n_batches = n_pairs > 0 ? batch + 1 : 0;
  return VGICP_OK;
}

}  // extern "C"
