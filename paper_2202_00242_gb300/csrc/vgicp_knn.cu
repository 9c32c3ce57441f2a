// Point covariances from k nearest neighbours (arXiv 2202.00242 Sec. III-C: each
// input point is modelled as a Gaussian whose covariance comes from its
// neighbouring points; GICP-style regularisation).
//
// For a batch of clouds given by offsets (neighbours are searched within each
// cloud only):
//   cell      per cloud, the grid cell size h: the caller's, or
//             sqrt(A / n * 2k) from the cloud's bounding box (A = the sum of the
//             box's face areas), a cell holding a few k points on a surface
//   insert    per point: exact cell key floor(x / h) (binary64 semantics),
//             open-addressing insert into the cloud's cell table, count
//   scan      cell offsets; scatter: the points in cell order (float4: x, y, z,
//             point index), so a cell's members are contiguous
//   query     per point, in cell order: the cells at Chebyshev ring distance
//             s = 0, 1, ... from its own, visited until the kept candidates all
//             lie within s h (any point beyond lies farther than s h).  The
//             order is (d^2, index) with d^2 = ((dx dx + dy dy) + dz dz) in
//             binary64 from the exact float-to-double differences.  The search
//             keeps the KMAX > k best by float32 d^2 (within 2^-21 of the
//             binary64 value), then sorts those by the binary64 order; it is
//             certified when the last kept float32 d^2, lowered by the bound,
//             still exceeds the k-th binary64 d^2 (else the point is searched
//             again in binary64 throughout).
//   covariance  mean of the k neighbours in binary64, their scatter in float32
//             about it, the eigenvector v of the smallest eigenvalue by cyclic
//             Jacobi (float32, on the trace-normalised matrix), and
//             C = V diag(1, 1, eps) V^T = I - (1 - eps) v v^T.
#include <cuda_runtime.h>

#include <algorithm>
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

struct __align__(16) CellSlot {
  unsigned long long key;
  uint32_t start;  // first member in the cell-ordered arrays
  uint32_t count;
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

// Per cloud (one CTA each): cell size h and float32(1 / h).
__global__ void cell_size_kernel(const float* __restrict__ pts, const int64_t* __restrict__ off,
                                 int32_t k, double cell, double* __restrict__ h_out,
                                 float* __restrict__ inv_out) {
  const int c = blockIdx.x;
  const int64_t a = off[c], b = off[c + 1];
  __shared__ float mn[3][kThreads], mx[3][kThreads];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (!(cell > 0.0))
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x)
      for (int d = 0; d < 3; ++d) {
        const float v = pts[3 * i + d];
        lo[d] = fminf(lo[d], v);
        hi[d] = fmaxf(hi[d], v);
      }
  for (int d = 0; d < 3; ++d) {
    mn[d][threadIdx.x] = lo[d];
    mx[d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        mn[d][threadIdx.x] = fminf(mn[d][threadIdx.x], mn[d][threadIdx.x + s]);
        mx[d][threadIdx.x] = fmaxf(mx[d][threadIdx.x], mx[d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double h = cell;
    if (!(h > 0.0)) {
      double e[3];
      for (int d = 0; d < 3; ++d) e[d] = b > a ? (double)mx[d][0] - (double)mn[d][0] : 1.0;
      const double area = fmax(e[0] * e[1] + e[1] * e[2] + e[0] * e[2], 1e-12);
      h = fmax(sqrt(area / (double)(b > a ? b - a : 1) * 2.0 * k), 1e-3);
    }
    h_out[c] = h;
    inv_out[c] = (float)(1.0 / h);
  }
}

__global__ void cell_init_kernel(CellSlot* slots, int64_t cap_total) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    CellSlot e;
    e.key = kEmptyKey;
    e.start = 0u;
    e.count = 0u;
    slots[s] = e;
  }
}

__device__ __forceinline__ void cell_key(const float* p, double h, float inv, int& kx, int& ky,
                                         int& kz) {
  kx = axis_key_target(p[0], inv, h);
  ky = axis_key_target(p[1], inv, h);
  kz = axis_key_target(p[2], inv, h);
}

__global__ void cell_insert_kernel(const float* __restrict__ pts, int64_t n,
                                   const int64_t* __restrict__ off, int32_t n_clouds,
                                   const double* __restrict__ hc, const float* __restrict__ invc,
                                   const int64_t* __restrict__ slot_base,
                                   const uint32_t* __restrict__ cap_mask, CellSlot* slots,
                                   uint32_t* __restrict__ pt_slot, int32_t* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = cloud_of(off, n_clouds, i);
    int kx, ky, kz;
    cell_key(pts + 3 * i, hc[c], invc[c], kx, ky, kz);
    if (!key_in_range(kx) || !key_in_range(ky) || !key_in_range(kz)) {
      pt_slot[i] = kNoSlot;
      set_status(status, VGICP_ERR_KEY_RANGE);
      continue;
    }
    const unsigned long long key = pack_key(kx, ky, kz);
    const uint32_t mask = cap_mask[c];
    CellSlot* t = slots + slot_base[c];
    uint32_t h = hash_key(kx, ky, kz) & mask;
    uint32_t found = kNoSlot;
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
      h = (h + 1) & mask;
    }
    if (found == kNoSlot) {
      pt_slot[i] = kNoSlot;
      set_status(status, VGICP_ERR_HASH_FULL);
      continue;
    }
    atomicAdd(&t[found].count, 1u);
    pt_slot[i] = (uint32_t)(slot_base[c] + found);
  }
}

__global__ void cell_counts_kernel(const CellSlot* __restrict__ slots, int64_t cap_total,
                                   uint32_t* __restrict__ cnt) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap_total;
       s += (int64_t)gridDim.x * blockDim.x)
    cnt[s] = slots[s].count;
}

__global__ void cell_starts_kernel(CellSlot* slots, int64_t cap_total,
                                   const uint32_t* __restrict__ start, uint32_t* __restrict__ fill) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < cap_total;
       s += (int64_t)gridDim.x * blockDim.x) {
    slots[s].start = start[s];
    fill[s] = 0u;
  }
}

__global__ void cell_scatter_kernel(const float* __restrict__ pts, int64_t n,
                                    const uint32_t* __restrict__ pt_slot,
                                    const CellSlot* __restrict__ slots, uint32_t* fill,
                                    float4* __restrict__ members) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = pt_slot[i];
    if (s == kNoSlot) continue;
    const uint32_t pos = slots[s].start + atomicAdd(fill + s, 1u);
    members[pos] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2],
                               __uint_as_float((uint32_t)i));
  }
}

// Candidate order: (d^2, index), lexicographic.  Non-negative binary64 values
// order like their bit patterns read as unsigned integers, so the comparison
// runs on the integer pipe (binary64 arithmetic is scarce on this GPU).
__device__ __forceinline__ bool before(unsigned long long d, uint32_t j, unsigned long long e,
                                       uint32_t l) {
  return d < e || (d == e && j < l);
}

// Smallest-eigenvalue eigenvector of a symmetric 3x3 matrix (upper triangle a)
// by cyclic Jacobi rotations (float32).
__device__ void smallest_eigvec(const float a_in[6], float v_out[3]) {
  float A[3][3] = {{a_in[0], a_in[1], a_in[2]}, {a_in[1], a_in[3], a_in[4]},
                   {a_in[2], a_in[4], a_in[5]}};
  float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  for (int sweep = 0; sweep < 12; ++sweep) {
    const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
    if (off < 1e-12f * (fabsf(A[0][0]) + fabsf(A[1][1]) + fabsf(A[2][2])) || off == 0.f) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      const float apq = A[p][q];
      if (apq == 0.f) continue;
      const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
      const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      const float c = rsqrtf(t * t + 1.f), s = t * c;
#pragma unroll
      for (int r = 0; r < 3; ++r) {  // A <- A J
        const float arp = A[r][p], arq = A[r][q];
        A[r][p] = c * arp - s * arq;
        A[r][q] = s * arp + c * arq;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {  // A <- J^T A
        const float apr = A[p][r], aqr = A[q][r];
        A[p][r] = c * apr - s * aqr;
        A[q][r] = s * apr + c * aqr;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {  // V <- V J
        const float vrp = V[r][p], vrq = V[r][q];
        V[r][p] = c * vrp - s * vrq;
        V[r][q] = s * vrp + c * vrq;
      }
    }
  }
  int m = 0;
  if (A[1][1] < A[m][m]) m = 1;
  if (A[2][2] < A[m][m]) m = 2;
  float n2 = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    v_out[r] = V[r][m];
    n2 += v_out[r] * v_out[r];
  }
  const float s = rsqrtf(n2);
#pragma unroll
  for (int r = 0; r < 3; ++r) v_out[r] *= s;
}

// Candidate order in float32: (f2, index), lexicographic.
__device__ __forceinline__ bool before_f(float d, uint32_t j, float e, uint32_t l) {
  return d < e || (d == e && j < l);
}

// Visits the cells of ring s around (cx, cy, cz); for each member calls f(q).
template <typename F>
__device__ __forceinline__ void for_ring(int s, int cx, int cy, int cz, uint32_t mask,
                                         const CellSlot* __restrict__ t,
                                         const float4* __restrict__ members, int64_t& seen,
                                         F&& f) {
  for (int dz = -s; dz <= s; ++dz)
    for (int dy = -s; dy <= s; ++dy)
      for (int dx = -s; dx <= s; ++dx) {
        if (max(abs(dx), max(abs(dy), abs(dz))) != s) continue;
        const int kx = cx + dx, ky = cy + dy, kz = cz + dz;
        if (!key_in_range(kx) || !key_in_range(ky) || !key_in_range(kz)) continue;
        const unsigned long long key = pack_key(kx, ky, kz);
        uint32_t hh = hash_key(kx, ky, kz) & mask;
        int found = -1;
        for (int p = 0; p < kMaxProbe; ++p) {
          const unsigned long long cur = t[hh].key;
          if (cur == key) {
            found = (int)hh;
            break;
          }
          if (cur == kEmptyKey) break;
          hh = (hh + 1) & mask;
        }
        if (found < 0) continue;
        const uint32_t s0 = t[found].start, cnt = t[found].count;
        seen += cnt;
        for (uint32_t m = 0; m < cnt; ++m) f(members[s0 + m]);
      }
}

// Exact k nearest (binary64 (d^2, index) order) by the ring search, for the rare
// points whose float32 pass cannot certify its result.  bd/bi: KMAX entries,
// the k best last (KMAX - k sentinels (0, 0) in front).
template <int KMAX>
__device__ __noinline__ void knn_exact(float px, float py, float pz, int cx, int cy, int cz,
                                       int k, int64_t nc, double h, uint32_t mask,
                                       const CellSlot* __restrict__ t,
                                       const float4* __restrict__ members,
                                       unsigned long long* bd, uint32_t* bi, int& held_out) {
  const double dpx = px, dpy = py, dpz = pz;
  for (int a = 0; a < KMAX; ++a) {
    const bool sentinel = a < KMAX - k;
    bd[a] = sentinel ? 0ull : 0x7FF0000000000000ull;
    bi[a] = sentinel ? 0u : 0xFFFFFFFFu;
  }
  const int64_t want = nc < (int64_t)k ? nc : (int64_t)k;
  int64_t held = 0, seen = 0;
  for (int s = 0;; ++s) {
    for_ring(s, cx, cy, cz, mask, t, members, seen, [&](const float4 q) {
      const double ex = __dsub_rn((double)q.x, dpx), ey = __dsub_rn((double)q.y, dpy),
                   ez = __dsub_rn((double)q.z, dpz);
      const unsigned long long d2 = (unsigned long long)__double_as_longlong(
          __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
      const uint32_t j = __float_as_uint(q.w);
      if (!before(d2, j, bd[KMAX - 1], bi[KMAX - 1])) return;
      int a = KMAX - 1;
      while (a > 0 && before(d2, j, bd[a - 1], bi[a - 1])) {
        bd[a] = bd[a - 1];
        bi[a] = bi[a - 1];
        --a;
      }
      bd[a] = d2;
      bi[a] = j;
      if (held < k) ++held;
    });
    const double reach = (double)s * h;
    if (held >= want && (held == 0 || __longlong_as_double((long long)bd[KMAX - 1]) < reach * reach))
      break;
    if (seen >= nc) break;
  }
  held_out = (int)held;
}

// Float32 squared distance relative to the binary64 one: within 2^-21 (the
// differences and the fused sum each round once; see the bound in the text).
constexpr float kF2Lo = 0.99999809265136719f;  // 1 - 2^-19
constexpr float kF2Hi = 1.0000019073486328f;   // 1 + 2^-19

template <int KMAX>
__global__ void __launch_bounds__(kThreads) knn_query_kernel(
    const float* __restrict__ pts, int64_t n, const int64_t* __restrict__ off, int32_t n_clouds,
    int32_t k, float eps, const double* __restrict__ hc, const float* __restrict__ invc,
    const int64_t* __restrict__ slot_base, const uint32_t* __restrict__ cap_mask,
    const CellSlot* __restrict__ slots, const float4* __restrict__ members,
    int32_t* __restrict__ nbr_out, float* __restrict__ covs_out) {
  // queries in cell order: the lanes of a warp search the same few cells
  for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < n;
       pos += (int64_t)gridDim.x * blockDim.x) {
    const float4 me = members[pos];
    const int64_t i = __float_as_uint(me.w);
    if (i >= n) continue;  // unfilled entry (a point without a cell: status is set)
    const int c = cloud_of(off, n_clouds, i);
    const int64_t base = off[c], nc = off[c + 1] - base;
    const double h = hc[c];
    const float px = me.x, py = me.y, pz = me.z;
    int cx, cy, cz;
    cell_key(pts + 3 * i, h, invc[c], cx, cy, cz);
    const uint32_t mask = cap_mask[c];
    const CellSlot* t = slots + slot_base[c];
    // 1. float32 pass: the KMAX best by (f2, index), all real entries
    float bf[KMAX];
    uint32_t bi[KMAX];
#pragma unroll
    for (int a = 0; a < KMAX; ++a) {
      bf[a] = INFINITY;
      bi[a] = 0xFFFFFFFFu;
    }
    const int64_t want = nc < (int64_t)KMAX ? nc : (int64_t)KMAX;
    int64_t held = 0, seen = 0;
    for (int s = 0;; ++s) {
      for_ring(s, cx, cy, cz, mask, t, members, seen, [&](const float4 q) {
        const float fx = q.x - px, fy = q.y - py, fz = q.z - pz;
        const float f2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        const uint32_t j = __float_as_uint(q.w);
        if (!before_f(f2, j, bf[KMAX - 1], bi[KMAX - 1])) return;
        bf[KMAX - 1] = f2;
        bi[KMAX - 1] = j;
#pragma unroll
        for (int a = KMAX - 1; a > 0; --a) {
          if (before_f(bf[a], bi[a], bf[a - 1], bi[a - 1])) {
            const float tf = bf[a];
            bf[a] = bf[a - 1];
            bf[a - 1] = tf;
            const uint32_t ti = bi[a];
            bi[a] = bi[a - 1];
            bi[a - 1] = ti;
          }
        }
        if (held < KMAX) ++held;
      });
      // every point not yet visited lies farther than s h
      const float reach2 = __double2float_rd((double)s * h * ((double)s * h));
      if (held >= want && bf[KMAX - 1] * kF2Hi < reach2) break;
      if (seen >= nc) break;
    }
    // 2. binary64 distances of the kept candidates, sorted exactly
    unsigned long long bd[KMAX];
#pragma unroll
    for (int a = 0; a < KMAX; ++a) {
      if (a < held) {
        const int64_t j = bi[a];
        const double ex = __dsub_rn((double)pts[3 * j], (double)px),
                     ey = __dsub_rn((double)pts[3 * j + 1], (double)py),
                     ez = __dsub_rn((double)pts[3 * j + 2], (double)pz);
        bd[a] = (unsigned long long)__double_as_longlong(
            __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
      } else {
        bd[a] = 0x7FF0000000000000ull;
      }
    }
#pragma unroll
    for (int a = 1; a < KMAX; ++a)  // insertion network (the float32 order is nearly right)
#pragma unroll
      for (int b = a; b > 0; --b)
        if (before(bd[b], bi[b], bd[b - 1], bi[b - 1])) {
          const unsigned long long td = bd[b];
          bd[b] = bd[b - 1];
          bd[b - 1] = td;
          const uint32_t ti = bi[b];
          bi[b] = bi[b - 1];
          bi[b - 1] = ti;
        }
    // 3. certificate: every candidate left out (f2 >= the last kept f2) has a
    //    binary64 d^2 above the k-th kept one, unless all were kept
    int cnt = (int)(held < k ? held : k);
    bool exact_ok = held < KMAX;  // fewer than KMAX candidates in all: all kept
    if (!exact_ok) {
      double kth = 0.0;
#pragma unroll
      for (int a = 0; a < KMAX; ++a)
        if (a == k - 1) kth = __longlong_as_double((long long)bd[a]);
      exact_ok = (double)(bf[KMAX - 1] * kF2Lo) > kth;
    }
    if (!exact_ok) {
      unsigned long long ed[32];
      uint32_t ei[32];
      int h2 = 0;
      knn_exact<32>(px, py, pz, cx, cy, cz, k, nc, h, mask, t, members, ed, ei, h2);
      cnt = h2;
      for (int a = 0; a < KMAX; ++a) bi[a] = 0xFFFFFFFFu;
      for (int a = 0; a < k && a < KMAX; ++a) bi[a] = ei[32 - k + a];
    }
    // neighbours (cloud-local) and the regularised covariance
    if (nbr_out)
      for (int a = 0; a < k; ++a) {
        int32_t v = -1;
#pragma unroll
        for (int b = 0; b < KMAX; ++b)
          if (b == a && a < cnt) v = (int32_t)((int64_t)bi[b] - base);
        nbr_out[(int64_t)k * i + a] = v;
      }
    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
    for (int b = 0; b < KMAX; ++b)
      if (b < cnt) {
        const int64_t j = bi[b];
        m0 += pts[3 * j] - px;
        m1 += pts[3 * j + 1] - py;
        m2 += pts[3 * j + 2] - pz;
      }
    const float idn = cnt > 0 ? 1.0f / (float)cnt : 0.f;
    m0 *= idn;
    m1 *= idn;
    m2 *= idn;
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < KMAX; ++b)
      if (b < cnt) {
        const int64_t j = bi[b];
        const float e0 = (pts[3 * j] - px) - m0, e1 = (pts[3 * j + 1] - py) - m1,
                    e2 = (pts[3 * j + 2] - pz) - m2;
        S[0] = fmaf(e0, e0, S[0]);
        S[1] = fmaf(e0, e1, S[1]);
        S[2] = fmaf(e0, e2, S[2]);
        S[3] = fmaf(e1, e1, S[3]);
        S[4] = fmaf(e1, e2, S[4]);
        S[5] = fmaf(e2, e2, S[5]);
      }
    const float tr = S[0] + S[3] + S[5];
    float v[3] = {0.f, 0.f, 1.f};
    if (tr > 0.f) {
      const float itr = 1.0f / tr;
      float a6[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) a6[r] = S[r] * itr;
      smallest_eigvec(a6, v);
    }
    const float w = 1.0f - eps;
    float* o = covs_out + 6 * i;
    o[0] = 1.0f - w * v[0] * v[0];
    o[1] = -w * v[0] * v[1];
    o[2] = -w * v[0] * v[2];
    o[3] = 1.0f - w * v[1] * v[1];
    o[4] = -w * v[1] * v[2];
    o[5] = 1.0f - w * v[2] * v[2];
  }
}

int grid_of(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 0x7FFFFFFF));
}

}  // namespace
}  // namespace vgicp

extern "C" {

int vgicp_estimate_covariances(const float* points, const int64_t* offsets, int32_t n_clouds,
                               int32_t k, double eps, double cell, int32_t* nbr_out,
                               float* covs_out, vgicp_stream_t stream) {
  using namespace vgicp;
  if (n_clouds <= 0 || !offsets) return set_error(VGICP_ERR_INVALID_ARG, "n_clouds must be >= 1");
  if (k < 1 || k > 32) return set_error(VGICP_ERR_INVALID_ARG, "k must be in [1, 32]");
  if (!(eps > 0.0) || eps > 1.0) return set_error(VGICP_ERR_INVALID_ARG, "eps must be in (0, 1]");
  if (!(cell >= 0.0) || !std::isfinite(cell))
    return set_error(VGICP_ERR_INVALID_ARG, "cell must be 0 (automatic) or positive");
  if (offsets[0] != 0) return set_error(VGICP_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (int32_t c = 0; c < n_clouds; ++c)
    if (offsets[c + 1] < offsets[c])
      return set_error(VGICP_ERR_INVALID_ARG, "offsets must be non-decreasing");
  const int64_t n = offsets[n_clouds];
  if (n >= (int64_t)0xFFFFFFFFll) return set_error(VGICP_ERR_INVALID_ARG, "more than 2^32-1 points");
  if (n == 0) return VGICP_OK;
  int rc = check_cloud(points, covs_out, n, "cloud");
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // per-cloud cell tables: capacity next_pow2(2 n_c)
  std::vector<int64_t> base((size_t)n_clouds);
  std::vector<uint32_t> mask((size_t)n_clouds);
  int64_t cap_total = 0;
  for (int32_t c = 0; c < n_clouds; ++c) {
    uint64_t cap = 16;
    while (cap < 2ull * (uint64_t)std::max<int64_t>(offsets[c + 1] - offsets[c], 1)) cap <<= 1;
    base[(size_t)c] = cap_total;
    mask[(size_t)c] = (uint32_t)(cap - 1);
    cap_total += (int64_t)cap;
  }
  if (cap_total >= (int64_t)0xFFFFFFFFll)
    return set_error(VGICP_ERR_INVALID_ARG, "more than 2^32-1 cell slots");
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
    return o;
  };
  const size_t o_off = take(sizeof(int64_t) * (n_clouds + 1));
  const size_t o_base = take(sizeof(int64_t) * n_clouds);
  const size_t o_mask = take(sizeof(uint32_t) * n_clouds);
  const size_t o_h = take(sizeof(double) * n_clouds);
  const size_t o_inv = take(sizeof(float) * n_clouds);
  const size_t o_status = take(sizeof(int32_t));
  const size_t o_slots = take(sizeof(CellSlot) * cap_total);
  const size_t o_ptslot = take(sizeof(uint32_t) * n);
  const size_t o_cnt = take(sizeof(uint32_t) * cap_total);
  const size_t o_start = take(sizeof(uint32_t) * cap_total);
  const size_t o_members = take(sizeof(float4) * n);
  const size_t o_scan = take(sizeof(uint32_t) * scan_tmp_elems(cap_total));
  char* d = nullptr;
  VGICP_CUDA_TRY(device_malloc(reinterpret_cast<void**>(&d), off, st, true));
  auto P = [&](size_t o) { return d + o; };
  int64_t* d_off = reinterpret_cast<int64_t*>(P(o_off));
  int64_t* d_base = reinterpret_cast<int64_t*>(P(o_base));
  uint32_t* d_mask = reinterpret_cast<uint32_t*>(P(o_mask));
  double* d_h = reinterpret_cast<double*>(P(o_h));
  float* d_inv = reinterpret_cast<float*>(P(o_inv));
  int32_t* d_status = reinterpret_cast<int32_t*>(P(o_status));
  CellSlot* d_slots = reinterpret_cast<CellSlot*>(P(o_slots));
  uint32_t* d_ptslot = reinterpret_cast<uint32_t*>(P(o_ptslot));
  uint32_t* d_cnt = reinterpret_cast<uint32_t*>(P(o_cnt));
  uint32_t* d_start = reinterpret_cast<uint32_t*>(P(o_start));
  float4* d_members = reinterpret_cast<float4*>(P(o_members));
  uint32_t* d_scan = reinterpret_cast<uint32_t*>(P(o_scan));
  // (copies from pageable memory return once the source is staged)
  cudaError_t e = cudaMemcpyAsync(d_off, offsets, sizeof(int64_t) * (n_clouds + 1),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * n_clouds, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_mask, mask.data(), sizeof(uint32_t) * n_clouds, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_members, 0xFF, sizeof(float4) * n, st);
  if (e != cudaSuccess) rc = check_cuda(e, "estimate_covariances setup");
  if (rc == VGICP_OK) {
    const int g = grid_of(n), gs = grid_of(cap_total);
    cell_size_kernel<<<n_clouds, kThreads, 0, st>>>(points, d_off, k, cell, d_h, d_inv);
    cell_init_kernel<<<gs, kThreads, 0, st>>>(d_slots, cap_total);
    cell_insert_kernel<<<g, kThreads, 0, st>>>(points, n, d_off, n_clouds, d_h, d_inv, d_base,
                                               d_mask, d_slots, d_ptslot, d_status);
    cell_counts_kernel<<<gs, kThreads, 0, st>>>(d_slots, cap_total, d_cnt);
    count_launches(4);
    rc = launch_exclusive_scan(d_cnt, d_start, cap_total, nullptr, d_scan, nullptr, st);
    if (rc == VGICP_OK) {
      cell_starts_kernel<<<gs, kThreads, 0, st>>>(d_slots, cap_total, d_start, d_cnt);
      cell_scatter_kernel<<<g, kThreads, 0, st>>>(points, n, d_ptslot, d_slots, d_cnt, d_members);
      if (k <= 12)
        knn_query_kernel<16><<<g, kThreads, 0, st>>>(points, n, d_off, n_clouds, k, (float)eps,
                                                     d_h, d_inv, d_base, d_mask, d_slots,
                                                     d_members, nbr_out, covs_out);
      else
        knn_query_kernel<32><<<g, kThreads, 0, st>>>(points, n, d_off, n_clouds, k, (float)eps,
                                                     d_h, d_inv, d_base, d_mask, d_slots,
                                                     d_members, nbr_out, covs_out);
      count_launches(3);
      e = cudaGetLastError();
      if (e != cudaSuccess) rc = check_cuda(e, "estimate_covariances kernels");
    }
  }
  int32_t status = 0;
  if (rc == VGICP_OK) {
    e = cudaMemcpyAsync(&status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = check_cuda(e, "estimate_covariances status");
  }
  e = cudaFreeAsync(d, st);
  if (rc == VGICP_OK && e != cudaSuccess) rc = check_cuda(e, "cudaFreeAsync");
  if (rc == VGICP_OK && status == VGICP_ERR_KEY_RANGE)
    rc = set_error(status, "a point's cell key is outside [-2^20, 2^20) (cell too small for "
                           "the coordinates, or not finite)");
  else if (rc == VGICP_OK && status == VGICP_ERR_HASH_FULL)
    rc = set_error(status, "cell table probe limit exceeded");
  return rc;
}

}  // extern "C"
