// Batched-linearization plans: the work list of a fixed factor set is built once,
// the launch shape is picked by timing candidates on the GPU (autotuner), and
// one linearization (pose upload, status reset, linearize, reduce) is captured
// in a CUDA graph that is replayed with new poses at every optimizer iteration
// (arXiv 2202.00242 Sec. III-A: the factors are re-linearized at every
// iteration; Sec. III-F: the global map links every overlapping submap pair).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "vgicp.h"
#include "vgicp_internal.h"
#include "vgicp_se3.cuh"

using namespace vgicp;

struct vgicp_plan {
  int device = 0;
  int32_t n_pairs = 0;
  std::vector<int32_t> pairs;    // 2 x n_pairs (map, source)
  std::vector<int64_t> src_n;    // points per source
  std::vector<MapDesc> md;
  std::vector<SrcDesc> sd;
  std::vector<int64_t> order;    // pairs sorted by (map, source)
  int32_t neighbours = 1;
  int32_t variant = 0, item = 0, grid = 0;  // current launch shape
  int64_t n_items = 0;
  int64_t items_cap = 0;
  // device
  char* d_block = nullptr;
  PairDesc* d_pd = nullptr;
  MapDesc* d_md = nullptr;
  SrcDesc* d_sd = nullptr;
  WorkItem* d_items = nullptr;
  int2* d_span = nullptr;
  int32_t* d_status = nullptr;
  double* d_partials = nullptr;
  double* d_out = nullptr;
  int64_t* d_inl = nullptr;
  int2* d_ms = nullptr;          // (map, source) of each pair
  double* d_jr = nullptr;        // right Jacobians of the last differentiable evaluation
  // host: two pinned staging buffers of the per-pair poses, used alternately;
  // uploaded[b] fires when the copy out of buffer b has completed
  PairDesc* h_pd[2] = {nullptr, nullptr};
  cudaEvent_t uploaded[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int next_buf = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kMinItem = 2048;

int build_items(vgicp_plan* P, int item) {
  std::vector<WorkItem> items;
  std::vector<int2> span((size_t)P->n_pairs);
  for (int64_t q = 0; q < P->n_pairs; ++q) {
    const int64_t p = P->order[(size_t)q];
    const int64_t n = P->src_n[(size_t)P->pairs[2 * p + 1]];
    const int32_t first = (int32_t)items.size();
    for (int64_t b = 0; b < n; b += item)
      items.push_back(WorkItem{(int32_t)p, (int32_t)b, (int32_t)std::min<int64_t>(n, b + item), 0});
    span[(size_t)p] = make_int2(first, (int32_t)items.size());
  }
  if ((int64_t)items.size() > P->items_cap)
    return set_error(VGICP_ERR_INVALID_ARG, "item size below the plan's minimum");
  P->n_items = (int64_t)items.size();
  P->item = item;
  if (!items.empty())
    VGICP_CUDA_TRY(cudaMemcpy(P->d_items, items.data(), sizeof(WorkItem) * items.size(),
                              cudaMemcpyHostToDevice));
  VGICP_CUDA_TRY(cudaMemcpy(P->d_span, span.data(), sizeof(int2) * span.size(),
                            cudaMemcpyHostToDevice));
  return VGICP_OK;
}

LinLaunch launch_of(const vgicp_plan* P) {
  LinLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.items = P->d_items;
  L.n_items = (int32_t)P->n_items;
  L.item_size = P->item;
  L.pairs = P->d_pd;
  L.maps = P->d_md;
  L.srcs = P->d_sd;
  L.partials = P->d_partials;
  L.status = P->d_status;
  L.neighbours = P->neighbours;
  L.variant = P->variant;
  L.grid = P->grid;
  return L;
}

// One linearization of the plan's factors on stream st (no pose upload).
int run_once(const vgicp_plan* P, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  VGICP_CUDA_TRY(cudaMemsetAsync(P->d_status, 0, 2 * sizeof(int32_t), st));
  LinLaunch L = launch_of(P);
  L.ev_start = e0;
  L.ev_stop = e1;
  int rc = launch_linearize(L, st);
  if (rc) return rc;
  return launch_reduce(P->d_partials, P->d_span, 0, P->n_pairs, P->d_status, P->d_out, P->d_inl,
                       st);
}

// Convert the poses into staging buffer b (after its previous copy completed).
int stage_poses(vgicp_plan* P, const double* poses, int b) {
  if (P->used[b]) VGICP_CUDA_TRY(cudaEventSynchronize(P->uploaded[b]));
  for (int64_t p = 0; p < P->n_pairs; ++p) {
    if (!finite_pose(poses + 16 * p))
      return set_error(VGICP_ERR_INVALID_ARG,
                       "pose " + std::to_string(p) + " is not a finite rigid transform");
    P->h_pd[b][p] = make_pair_desc(poses + 16 * p, P->pairs[2 * p], P->pairs[2 * p + 1]);
  }
  return VGICP_OK;
}

// Copies n 16-byte words from pinned host memory (addressable from the device)
// to device memory.
__global__ void copy_words_kernel(uint4* __restrict__ dst, const uint4* __restrict__ src,
                                  int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// The poses go to the device through a kernel that reads the pinned staging
// buffer, not through a copy engine: a host-to-device copy queued there would
// wait behind whatever large upload the caller has in flight (for instance the
// next step's clouds on another stream).
int upload_poses(vgicp_plan* P, int b, cudaStream_t st) {
  static_assert(sizeof(PairDesc) % 16 == 0, "PairDesc is a whole number of 16-B words");
  const int64_t words = (int64_t)sizeof(PairDesc) / 16 * P->n_pairs;
  const int grid = (int)std::min<int64_t>((words + 255) / 256, 1024);
  copy_words_kernel<<<std::max(grid, 1), 256, 0, st>>>(reinterpret_cast<uint4*>(P->d_pd),
                                                        reinterpret_cast<const uint4*>(P->h_pd[b]),
                                                        words);
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  VGICP_CUDA_TRY(cudaEventRecord(P->uploaded[b], st));
  P->used[b] = true;
  return VGICP_OK;
}

// Pose of every factor for a differentiable evaluation, in binary64 on the
// device: T_p = T0_p Exp(xi_p) (xi = null: T0_p), written as the factor's
// descriptor, and J_r(xi_p) when jr is given.  A base pose that is not a finite
// rigid transform, or a non-finite increment, sets the status word (all
// outputs of the evaluation become NaN) and uses the identity.
__global__ void compose_kernel(const double* __restrict__ base, const double* __restrict__ xi,
                               const int2* __restrict__ ms, int64_t n_pairs,
                               PairDesc* __restrict__ pd, double* __restrict__ jr,
                               int32_t* __restrict__ status) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  double T0[16], x[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, E[16], T[16];
  for (int i = 0; i < 16; ++i) T0[i] = base[16 * p + i];
  bool ok = se3::rigid(T0);
  if (xi)
    for (int i = 0; i < 6; ++i) {
      x[i] = xi[6 * p + i];
      ok = ok && isfinite(x[i]);
    }
  if (!ok) {
    atomicExch(status, 2);
    for (int i = 0; i < 16; ++i) T0[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int i = 0; i < 6; ++i) x[i] = 0.0;
  }
  se3::expmap(x, E);
  se3::pose_mul(T0, E, T);
  pd[p] = se3::pair_desc(T, ms[p].x, ms[p].y);
  if (jr) se3::right_jacobian(x, jr + 36 * p);
}

void drop_graph(vgicp_plan* P) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->exec = nullptr;
  P->graph = nullptr;
}

// Capture: status reset, linearize, reduce.  The pose upload stays outside the
// graph.
int capture_graph(vgicp_plan* P) {
  drop_graph(P);
  // a first launch outside capture sets per-kernel attributes
  int rc = run_once(P, P->cap, nullptr, nullptr);
  if (rc) return rc;
  VGICP_CUDA_TRY(cudaStreamSynchronize(P->cap));
  VGICP_CUDA_TRY(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeRelaxed));
  rc = run_once(P, P->cap, nullptr, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(P->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e2 != cudaSuccess) return check_cuda(e2, "cudaStreamEndCapture");
  P->graph = g;
  VGICP_CUDA_TRY(cudaGraphInstantiate(&P->exec, g, 0));
  return VGICP_OK;
}

void destroy_plan(vgicp_plan* P) {
  if (!P) return;
  drop_graph(P);
  for (int b = 0; b < 2; ++b) {
    if (P->uploaded[b]) cudaEventDestroy(P->uploaded[b]);
    if (P->h_pd[b]) cudaFreeHost(P->h_pd[b]);
  }
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->d_block) cudaFree(P->d_block);
  delete P;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

int vgicp_plan_create(vgicp_map* const* maps, int32_t n_maps, const vgicp_cloud* sources,
                      int32_t n_sources, const int32_t* pairs, int64_t n_pairs,
                      const vgicp_lin_opts* opts, vgicp_stream_t stream, vgicp_plan** out) {
  (void)stream;
  if (!out) return set_error(VGICP_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!maps || n_maps <= 0 || !sources || n_sources <= 0 || !pairs || n_pairs <= 0)
    return set_error(VGICP_ERR_INVALID_ARG, "empty or null plan arguments");
  if (n_pairs > INT32_MAX / 2) return set_error(VGICP_ERR_INVALID_ARG, "too many pairs");
  const int neighbours = opts && opts->neighbours ? opts->neighbours : 1;
  if (neighbours != 1 && neighbours != 27)
    return set_error(VGICP_ERR_INVALID_ARG, "neighbours must be 1 or 27");
  if (opts && (opts->variant < 0 || opts->variant > 3))
    return set_error(VGICP_ERR_INVALID_ARG, "variant must be 0, 1, 2 or 3");
  if (opts && (opts->corr_out || opts->qkey_out))
    return set_error(VGICP_ERR_INVALID_ARG, "corr_out/qkey_out are single-factor options");
  if (opts && opts->tile > 0 && opts->tile < kMinItem)
    return set_error(VGICP_ERR_INVALID_ARG, "plan item size must be at least 2048 points");
  vgicp_plan* P = new vgicp_plan();
  cudaGetDevice(&P->device);
  P->n_pairs = (int32_t)n_pairs;
  P->neighbours = neighbours;
  P->variant = opts ? opts->variant : 0;
  P->grid = opts ? opts->grid : 0;
  P->pairs.assign(pairs, pairs + 2 * n_pairs);
  for (int32_t m = 0; m < n_maps; ++m) {
    if (!maps[m]) {
      destroy_plan(P);
      return set_error(VGICP_ERR_INVALID_ARG, "null map handle");
    }
    P->md.push_back(make_map_desc(maps[m]));
  }
  for (int32_t c = 0; c < n_sources; ++c) {
    if (sources[c].map) {
      const vgicp_map* m = sources[c].map;
      const int64_t a = m->set->point_off[m->index], b = m->set->point_off[m->index + 1];
      P->sd.push_back(SrcDesc{m->set->d_gpts + 3 * a, m->set->d_gcovs + 6 * a, b - a});
    } else {
      int rc = check_cloud(sources[c].points, sources[c].covs, sources[c].n, "source cloud");
      if (rc) {
        destroy_plan(P);
        return rc;
      }
      P->sd.push_back(SrcDesc{sources[c].points, sources[c].covs, sources[c].n});
    }
    P->src_n.push_back(P->sd.back().n);
  }
  for (int64_t p = 0; p < n_pairs; ++p) {
    const int32_t m = pairs[2 * p], c = pairs[2 * p + 1];
    if (m < 0 || m >= n_maps || c < 0 || c >= n_sources) {
      destroy_plan(P);
      return set_error(VGICP_ERR_INVALID_ARG, "pair index out of range");
    }
    P->order.push_back(p);
  }
  std::stable_sort(P->order.begin(), P->order.end(), [&](int64_t a, int64_t b) {
    return pairs[2 * a] != pairs[2 * b] ? pairs[2 * a] < pairs[2 * b]
                                        : pairs[2 * a + 1] < pairs[2 * b + 1];
  });
  int64_t cap = 0;
  for (int64_t p = 0; p < n_pairs; ++p)
    cap += (P->src_n[(size_t)pairs[2 * p + 1]] + kMinItem - 1) / kMinItem;
  P->items_cap = std::max<int64_t>(cap, 1);
  if (P->items_cap > INT32_MAX / 2) {
    destroy_plan(P);
    return set_error(VGICP_ERR_INVALID_ARG, "too many work items");
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  const size_t o_pd = take(sizeof(PairDesc) * n_pairs);
  const size_t o_md = take(sizeof(MapDesc) * P->md.size());
  const size_t o_sd = take(sizeof(SrcDesc) * P->sd.size());
  const size_t o_items = take(sizeof(WorkItem) * P->items_cap);
  const size_t o_span = take(sizeof(int2) * n_pairs);
  const size_t o_status = take(sizeof(int32_t));
  const size_t o_part = take(sizeof(double) * kPartialStride * P->items_cap);
  const size_t o_out = take(sizeof(double) * 43 * n_pairs);
  const size_t o_inl = take(sizeof(int64_t) * n_pairs);
  const size_t o_ms = take(sizeof(int2) * n_pairs);
  const size_t o_jr = take(sizeof(double) * 36 * n_pairs);
  cudaError_t e = device_malloc(reinterpret_cast<void**>(&P->d_block), off, nullptr, false);
  if (e != cudaSuccess) {
    cudaGetLastError();
    destroy_plan(P);
    return set_error(VGICP_ERR_OOM, "plan allocation of " + std::to_string(off) + " bytes failed");
  }
  P->d_pd = reinterpret_cast<PairDesc*>(P->d_block + o_pd);
  P->d_md = reinterpret_cast<MapDesc*>(P->d_block + o_md);
  P->d_sd = reinterpret_cast<SrcDesc*>(P->d_block + o_sd);
  P->d_items = reinterpret_cast<WorkItem*>(P->d_block + o_items);
  P->d_span = reinterpret_cast<int2*>(P->d_block + o_span);
  P->d_status = reinterpret_cast<int32_t*>(P->d_block + o_status);
  P->d_partials = reinterpret_cast<double*>(P->d_block + o_part);
  P->d_out = reinterpret_cast<double*>(P->d_block + o_out);
  P->d_inl = reinterpret_cast<int64_t*>(P->d_block + o_inl);
  P->d_ms = reinterpret_cast<int2*>(P->d_block + o_ms);
  P->d_jr = reinterpret_cast<double*>(P->d_block + o_jr);
  std::vector<int2> ms((size_t)n_pairs);
  for (int64_t p = 0; p < n_pairs; ++p) ms[(size_t)p] = make_int2(pairs[2 * p], pairs[2 * p + 1]);
  int rc = VGICP_OK;
  if ((e = cudaMallocHost(&P->h_pd[0], sizeof(PairDesc) * n_pairs)) != cudaSuccess ||
      (e = cudaMallocHost(&P->h_pd[1], sizeof(PairDesc) * n_pairs)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&P->uploaded[0], cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&P->uploaded[1], cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMemcpy(P->d_ms, ms.data(), sizeof(int2) * ms.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(P->d_md, P->md.data(), sizeof(MapDesc) * P->md.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(P->d_sd, P->sd.data(), sizeof(SrcDesc) * P->sd.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    rc = check_cuda(e, "plan set-up");
  if (rc == VGICP_OK)
    rc = build_items(P, opts && opts->tile > 0 ? opts->tile : default_item_size());
  if (rc) {
    destroy_plan(P);
    return rc;
  }
  *out = P;
  return VGICP_OK;
}

int vgicp_plan_autotune(vgicp_plan* P, const double* poses, vgicp_stream_t stream) {
  if (!P || !poses) return set_error(VGICP_ERR_INVALID_ARG, "null plan or poses");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int buf = P->next_buf;
  P->next_buf ^= 1;
  int rc = stage_poses(P, poses, buf);
  if (rc) return rc;
  rc = upload_poses(P, buf, st);
  if (rc) return rc;
  VGICP_CUDA_TRY(cudaStreamSynchronize(st));
  const int variants_1[] = {1, 2, 3};
  const int variants_27[] = {1};
  const int* vs = P->neighbours == 27 ? variants_27 : variants_1;
  const int nv = P->neighbours == 27 ? 1 : (int)(sizeof(variants_1) / sizeof(variants_1[0]));
  const int items[] = {4096, 8192, 16384, 32768};
  float best = 1e30f;
  int best_v = 1, best_i = default_item_size();
  cudaEvent_t e0, e1;
  VGICP_CUDA_TRY(cudaEventCreate(&e0));
  VGICP_CUDA_TRY(cudaEventCreate(&e1));
  for (int a = 0; a < nv && rc == VGICP_OK; ++a) {
    for (int it : items) {
      P->variant = vs[a];
      if ((rc = build_items(P, it)) != VGICP_OK) break;
      if ((rc = run_once(P, st, nullptr, nullptr)) != VGICP_OK) break;  // warm-up
      float total = 0.f;
      for (int r = 0; r < 3 && rc == VGICP_OK; ++r) {
        rc = run_once(P, st, e0, e1);
        if (rc) break;
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = check_cuda(e, "autotune timing");
        total += ms;
      }
      if (rc == VGICP_OK && total < best) {
        best = total;
        best_v = vs[a];
        best_i = it;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  P->variant = best_v;
  rc = build_items(P, best_i);
  if (rc) return rc;
  drop_graph(P);
  return VGICP_OK;
}

int vgicp_plan_execute(vgicp_plan* P, const double* poses, double* out, int64_t* inliers,
                       void* kernel_start, void* kernel_stop, vgicp_stream_t stream) {
  if (!P || !poses) return set_error(VGICP_ERR_INVALID_ARG, "null plan or poses");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int buf = P->next_buf;
  P->next_buf ^= 1;
  int rc = stage_poses(P, poses, buf);
  if (rc) return rc;
  if (!P->exec) {
    // first execution: the graph is captured after this pose upload (the
    // capture stream waits for it)
    rc = upload_poses(P, buf, st);
    if (rc) return rc;
    VGICP_CUDA_TRY(cudaStreamSynchronize(st));
    rc = capture_graph(P);
    if (rc) return rc;
  } else {
    rc = upload_poses(P, buf, st);
    if (rc) return rc;
  }
  if (kernel_start) VGICP_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(kernel_start), st));
  VGICP_CUDA_TRY(cudaGraphLaunch(P->exec, st));
  count_launches(2);  // linearize + reduce
  if (kernel_stop) VGICP_CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(kernel_stop), st));
  if (out)
    VGICP_CUDA_TRY(cudaMemcpyAsync(out, P->d_out, sizeof(double) * 43 * P->n_pairs,
                                   cudaMemcpyDeviceToDevice, st));
  if (inliers)
    VGICP_CUDA_TRY(cudaMemcpyAsync(inliers, P->d_inl, sizeof(int64_t) * P->n_pairs,
                                   cudaMemcpyDeviceToDevice, st));
  return VGICP_OK;
}

int vgicp_plan_evaluate(vgicp_plan* P, const double* base_poses, const double* xi, int32_t mode,
                        const double* grad_scale, double* out, int64_t* inliers,
                        vgicp_stream_t stream) {
  if (!P || !base_poses || !out) return set_error(VGICP_ERR_INVALID_ARG, "null plan, poses or out");
  if (mode < 1 || mode > 3) return set_error(VGICP_ERR_INVALID_ARG, "mode must be 1, 2 or 3");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  VGICP_CUDA_TRY(cudaMemsetAsync(P->d_status, 0, 2 * sizeof(int32_t), st));
  double* jr = mode >= 2 && xi ? P->d_jr : nullptr;
  const int64_t n = P->n_pairs;
  compose_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(base_poses, xi, P->d_ms, n, P->d_pd,
                                                              jr, P->d_status);
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  LinLaunch L = launch_of(P);
  L.mode = mode;
  int rc = launch_linearize(L, st);
  if (rc) return rc;
  // the caller's inlier buffer, or the plan's own
  return launch_reduce(P->d_partials, P->d_span, 0, n, P->d_status, out,
                       inliers ? inliers : P->d_inl, st, mode, jr, grad_scale);
}

int vgicp_plan_info(const vgicp_plan* P, int32_t* variant, int32_t* item_points, int32_t* grid,
                    int64_t* n_items) {
  if (!P) return set_error(VGICP_ERR_INVALID_ARG, "null plan");
  if (variant) *variant = P->variant ? P->variant : default_variant();
  if (item_points) *item_points = P->item;
  if (grid)
    *grid = P->grid ? P->grid : std::min<int64_t>(linearize_grid(P->neighbours, P->variant),
                                                  P->n_items);
  if (n_items) *n_items = P->n_items;
  return VGICP_OK;
}

int vgicp_plan_destroy(vgicp_plan* P) {
  if (P) {
    for (int b = 0; b < 2; ++b)
      if (P->used[b]) cudaEventSynchronize(P->uploaded[b]);
    cudaDeviceSynchronize();  // no queued graph may still read the plan's buffers
    destroy_plan(P);
  }
  return VGICP_OK;
}

}  // extern "C"
