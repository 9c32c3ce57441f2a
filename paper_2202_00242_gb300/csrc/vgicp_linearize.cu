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
//   M'   = R^T C'_v R + C_k,  W' = M'^-1  (= R^T W R, symmetric adjugate / det)
//   u    = W' d'
//   err += d'^T u
//   b   += [ u x mu ; -u ]
//   H   += [[ [mu]x^T W' [mu]x , [mu]x W' ], [ ., W' ]]
// The 28 unique terms and the inlier count are accumulated per thread in
// float32, reduced across the warp in float32, across warps in binary64, and
// written as one binary64 partial per work item; a second kernel sums each
// pair's partials in item order.  The result is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "vgicp_device.cuh"
#include "vgicp_internal.h"

namespace vgicp {
namespace {

constexpr int kLinThreads = 256;

struct Pose32 {
  float R[9];
  float t[3];
  float tmax;
};

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
    const double dxp = x, dyp = y, dzp = z;
    int* kk[3] = {&kx, &ky, &kz};
    const bool amb[3] = {ax, ay, az};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!amb[a]) continue;
      double s = __dmul_rn(pd->R64[3 * a + 0], dxp);
      s = __dadd_rn(s, __dmul_rn(pd->R64[3 * a + 1], dyp));
      s = __dadd_rn(s, __dmul_rn(pd->R64[3 * a + 2], dzp));
      s = __dadd_rn(s, pd->t64[a]);
      double k = floor(__ddiv_rn(s, md.r));
      k = fmin(fmax(k, -2147483648.0), 2147483647.0);
      *kk[a] = (int)k;
    }
  }
}

__device__ __forceinline__ int lookup(const MapDesc& md, int kx, int ky, int kz) {
  if (!key_in_range(kx) || !key_in_range(ky) || !key_in_range(kz)) return -1;
  const unsigned long long key = pack_key(kx, ky, kz);
  const ulonglong2* slots = reinterpret_cast<const ulonglong2*>(md.slots);
  uint32_t h = hash_key(kx, ky, kz) & md.mask;
  for (int p = 0; p < md.max_probe; ++p) {
    const ulonglong2 s = __ldg(slots + h);
    if (s.x == key) return (int)(uint32_t)s.y;
    if (s.x == kEmptyKey) return -1;
    h = (h + 1) & md.mask;
  }
  return -1;
}

// Accumulator layout (float):
//   0..5   H_ww (00 01 02 11 12 22)      6..14 H_wv (row-major, w rows, v cols)
//   15..20 H_vv (00 01 02 11 12 22)      21..23 b_w   24..26 b_v   27 err
//   28     inlier count
__device__ __forceinline__ void add_term(float* acc, const Pose32& P, float x, float y, float z,
                                         const float* c, float qx, float qy, float qz,
                                         const float4 r0, const float4 r1, const float4 r2) {
  const float* R = P.R;
  // residual in the target frame, then rotated into the source frame
  const float tx = r0.x - qx, ty = r0.y - qy, tz = r0.z - qz;
  const float d0 = fmaf(R[0], tx, fmaf(R[3], ty, R[6] * tz));
  const float d1 = fmaf(R[1], tx, fmaf(R[4], ty, R[7] * tz));
  const float d2 = fmaf(R[2], tx, fmaf(R[5], ty, R[8] * tz));
  // voxel covariance C' (symmetric)
  const float v00 = r1.x, v01 = r1.y, v02 = r1.z, v11 = r1.w, v12 = r2.x, v22 = r2.y;
  // A = C' R
  const float a00 = fmaf(v00, R[0], fmaf(v01, R[3], v02 * R[6]));
  const float a01 = fmaf(v00, R[1], fmaf(v01, R[4], v02 * R[7]));
  const float a02 = fmaf(v00, R[2], fmaf(v01, R[5], v02 * R[8]));
  const float a10 = fmaf(v01, R[0], fmaf(v11, R[3], v12 * R[6]));
  const float a11 = fmaf(v01, R[1], fmaf(v11, R[4], v12 * R[7]));
  const float a12 = fmaf(v01, R[2], fmaf(v11, R[5], v12 * R[8]));
  const float a20 = fmaf(v02, R[0], fmaf(v12, R[3], v22 * R[6]));
  const float a21 = fmaf(v02, R[1], fmaf(v12, R[4], v22 * R[7]));
  const float a22 = fmaf(v02, R[2], fmaf(v12, R[5], v22 * R[8]));
  // M' = R^T A + C_k (upper triangle)
  const float m00 = fmaf(R[0], a00, fmaf(R[3], a10, fmaf(R[6], a20, c[0])));
  const float m01 = fmaf(R[0], a01, fmaf(R[3], a11, fmaf(R[6], a21, c[1])));
  const float m02 = fmaf(R[0], a02, fmaf(R[3], a12, fmaf(R[6], a22, c[2])));
  const float m11 = fmaf(R[1], a01, fmaf(R[4], a11, fmaf(R[7], a21, c[3])));
  const float m12 = fmaf(R[1], a02, fmaf(R[4], a12, fmaf(R[7], a22, c[4])));
  const float m22 = fmaf(R[2], a02, fmaf(R[5], a12, fmaf(R[8], a22, c[5])));
  // W' = adj(M') / det(M')
  const float i00 = fmaf(m11, m22, -m12 * m12);
  const float i01 = fmaf(m02, m12, -m01 * m22);
  const float i02 = fmaf(m01, m12, -m02 * m11);
  const float i11 = fmaf(m00, m22, -m02 * m02);
  const float i12 = fmaf(m01, m02, -m00 * m12);
  const float i22 = fmaf(m00, m11, -m01 * m01);
  const float det = fmaf(m00, i00, fmaf(m01, i01, m02 * i02));
  const float s = __frcp_rn(det);
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
  acc[28] += 1.0f;
}

template <int NEIGH>
__global__ void __launch_bounds__(kLinThreads, 2)
    linearize_kernel(const __grid_constant__ LinLaunch L) {
  __shared__ float red[kLinThreads / 32][kAcc];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int it = blockIdx.x; it < L.n_items; it += gridDim.x) {
    int pair, begin, end;
    if (L.items) {
      const WorkItem w = L.items[it];
      pair = w.pair;
      begin = w.begin;
      end = w.end;
    } else {
      pair = 0;
      begin = it * L.tile;
      end = (int)min((int64_t)begin + L.tile, L.single_src.n);
    }
    const PairDesc* pd = L.pairs ? L.pairs + pair : &L.single;
    Pose32 P;
#pragma unroll
    for (int k = 0; k < 9; ++k) P.R[k] = pd->R[k];
    P.t[0] = pd->t[0];
    P.t[1] = pd->t[1];
    P.t[2] = pd->t[2];
    P.tmax = pd->tmax;
    const MapDesc md = L.maps ? L.maps[pd->map] : L.single_map;
    const SrcDesc sd = L.srcs ? L.srcs[pd->src] : L.single_src;
    uint32_t vbase = 0;
    if (L.corr_out) vbase = *md.vbase;

    float acc[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k] = 0.0f;

    for (int p = begin + threadIdx.x; p < end; p += blockDim.x) {
      const float* pt = sd.pts + 3 * (int64_t)p;
      const float x = __ldg(pt + 0), y = __ldg(pt + 1), z = __ldg(pt + 2);
      const float2* cv = reinterpret_cast<const float2*>(sd.covs + 6 * (int64_t)p);
      const float2 c01 = __ldg(cv + 0), c23 = __ldg(cv + 1), c45 = __ldg(cv + 2);
      const float c[6] = {c01.x, c01.y, c23.x, c23.y, c45.x, c45.y};
      const float qx = fmaf(P.R[0], x, fmaf(P.R[1], y, fmaf(P.R[2], z, P.t[0])));
      const float qy = fmaf(P.R[3], x, fmaf(P.R[4], y, fmaf(P.R[5], z, P.t[1])));
      const float qz = fmaf(P.R[6], x, fmaf(P.R[7], y, fmaf(P.R[8], z, P.t[2])));
      int kx, ky, kz;
      source_key(P, pd, md, x, y, z, qx, qy, qz, kx, ky, kz);
      if (NEIGH == 1) {
        const int vid = lookup(md, kx, ky, kz);
        if (L.corr_out) L.corr_out[p] = vid < 0 ? -1 : (int)((uint32_t)vid - vbase);
        if (L.qkey_out) {
          L.qkey_out[3 * (int64_t)p + 0] = kx;
          L.qkey_out[3 * (int64_t)p + 1] = ky;
          L.qkey_out[3 * (int64_t)p + 2] = kz;
        }
        if (vid < 0) continue;
        const float4* rec = md.recs + 3 * (int64_t)vid;
        add_term(acc, P, x, y, z, c, qx, qy, qz, __ldg(rec), __ldg(rec + 1), __ldg(rec + 2));
      } else {
        if (L.corr_out) {
          const int own = lookup(md, kx, ky, kz);
          L.corr_out[p] = own < 0 ? -1 : (int)((uint32_t)own - vbase);
        }
        if (L.qkey_out) {
          L.qkey_out[3 * (int64_t)p + 0] = kx;
          L.qkey_out[3 * (int64_t)p + 1] = ky;
          L.qkey_out[3 * (int64_t)p + 2] = kz;
        }
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int vid = lookup(md, kx + dx, ky + dy, kz + dz);
              if (vid < 0) continue;
              const float4* rec = md.recs + 3 * (int64_t)vid;
              add_term(acc, P, x, y, z, c, qx, qy, qz, __ldg(rec), __ldg(rec + 1),
                       __ldg(rec + 2));
            }
      }
    }

    // warp: float32 butterfly; block: binary64 across warps
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
    __syncthreads();
    if (threadIdx.x < kAcc) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)red[w][threadIdx.x];
      L.partials[(int64_t)it * kPartialStride + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// One warp per pair: lane k sums term k over the pair's items in order.
__global__ void reduce_kernel(const double* __restrict__ partials,
                              const int32_t* __restrict__ item_off, int32_t n_items_single,
                              int64_t n_pairs, double* __restrict__ out,
                              int64_t* __restrict__ inliers) {
  const int64_t pair = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= n_pairs) return;
  const int32_t a = item_off ? item_off[pair] : 0;
  const int32_t b = item_off ? item_off[pair + 1] : n_items_single;
  double s = 0.0;
  if (lane < kAcc)
    for (int32_t it = a; it < b; ++it) s += partials[(int64_t)it * kPartialStride + lane];
  double* o = out + pair * 43;
  // H_ww (sym), H_wv / H_vw, H_vv (sym), b, err
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
    inliers[pair] = (int64_t)llrint(s);
  }
}

}  // namespace

int launch_linearize(const LinLaunch& L, cudaStream_t st) {
  if (L.n_items <= 0) return VGICP_OK;
  const int block = L.block > 0 ? L.block : kLinThreads;
  if (block != kLinThreads) return set_error(VGICP_ERR_INVALID_ARG, "unsupported block size");
  int grid = L.grid > 0 ? L.grid : device_sm_count() * 2;
  grid = std::min(grid, L.n_items);
  if (L.ev_start) VGICP_CUDA_TRY(cudaEventRecord(L.ev_start, st));
  if (L.neighbours == 27)
    linearize_kernel<27><<<grid, block, 0, st>>>(L);
  else
    linearize_kernel<1><<<grid, block, 0, st>>>(L);
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  if (L.ev_stop) VGICP_CUDA_TRY(cudaEventRecord(L.ev_stop, st));
  return VGICP_OK;
}

int launch_reduce(const double* partials, const int32_t* item_off, int32_t n_items_single,
                  int64_t n_pairs, double* out, int64_t* inliers, cudaStream_t st) {
  if (n_pairs <= 0) return VGICP_OK;
  const int warps = 8;
  const int64_t blocks = (n_pairs + warps - 1) / warps;
  reduce_kernel<<<(unsigned)blocks, warps * 32, 0, st>>>(partials, item_off, n_items_single,
                                                         n_pairs, out, inliers);
  VGICP_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return VGICP_OK;
}

}  // namespace vgicp
