// FP64 CPU oracle for VGICP matching-cost factor linearization.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
// restatement of what the GPU library computes.  It shares no code, header,
// table or constant with the CUDA path; only tests, the smoke check and the
// CPU-baseline leg of the benchmark may load it.  The product path never calls it.
//
// What it follows (arXiv 2202.00242, "Globally Consistent and Tightly Coupled 3D
// LiDAR Inertial Mapping"):
//   * Sec. III-A: each point p_k = (mu_k, C_k) is a Gaussian; the target cloud
//     P_j is discretised into voxels and each voxel holds the aggregate of the
//     means and covariances of its points.
//   * Eq. 2: e^M = sum over p_k in P_i of e^D2D(p_k, T).
//   * Eq. 3: e^D2D = d_k^T (C'_k + T C_k T^T)^-1 d_k, d_k = mu'_k - T mu_k, with
//     (mu'_k, C'_k) the voxel of P_j that contains T mu_k.
//   * Sec. III-A, last paragraph: the factor is re-linearised (derivatives of
//     Eq. 2 -> Hessian factor H, b) at the current linearisation point.
//   * Sec. III-C / III-D: point covariances come from the k nearest neighbours.
//   * Sec. III-D: overlap rate = fraction of P_i points that fall in a voxel of P_j
//     (the inlier count returned here, divided by |P_i|).
//
// Readings where the paper is silent (each is listed in the design notes):
//   * voxel key = floor((double)x / r) per axis (IEEE binary64 division, floor);
//   * "T C T^T" on a 3x3 covariance is read as R C R^T;
//   * voxel Gaussian = mean of the point means and mean of the point covariances,
//     sums taken in ascending point index, then divided by N;
//   * a source point whose voxel is empty contributes nothing and is not an inlier;
//   * linearisation variable: right perturbation T <- T Exp(xi), xi = [omega; v];
//     W is held at the linearisation point, so with J = d d_k / d xi,
//     H = sum J^T W J, b = sum J^T W d, err = sum d^T W d, and
//     err(xi) ~ err + 2 b^T xi + xi^T H xi;
//   * 27-neighbour mode: one independent term per occupied voxel among the
//     3x3x3 block around the point's voxel, offsets visited dz, dy, dx in -1..1.
//
// Everything is binary64; FP32 inputs are promoted.  Build with
// -ffp-contract=off so that x86 and Arm hosts round identically.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Key3 {
  int64_t x, y, z;
  bool operator==(const Key3& o) const { return x == o.x && y == o.y && z == o.z; }
  bool operator<(const Key3& o) const {
    return x != o.x ? x < o.x : (y != o.y ? y < o.y : z < o.z);
  }
};
struct Key3Hash {
  size_t operator()(const Key3& k) const {
    // Any mixing works here; std::unordered_map only needs consistency.
    uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)k.y * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)k.z * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// ---- 3x3 helpers on row-major double[9] -----------------------------------

void mat3_mul(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

void mat3_transpose(const double* A, double* At) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) At[3 * j + i] = A[3 * i + j];
}

// Symmetric matrix from the 6 upper-triangular entries xx, xy, xz, yy, yz, zz.
void sym_from_upper(const float* c, double* S) {
  S[0] = c[0]; S[1] = c[1]; S[2] = c[2];
  S[3] = c[1]; S[4] = c[3]; S[5] = c[4];
  S[6] = c[2]; S[7] = c[4]; S[8] = c[5];
}
void sym_from_upper_d(const double* c, double* S) {
  S[0] = c[0]; S[1] = c[1]; S[2] = c[2];
  S[3] = c[1]; S[4] = c[3]; S[5] = c[4];
  S[6] = c[2]; S[7] = c[4]; S[8] = c[5];
}

// Inverse of a 3x3 matrix by Gauss-Jordan elimination with partial pivoting.
// Returns false if a pivot is exactly zero.
bool mat3_inverse(const double* A, double* Ainv) {
  double a[3][6];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) a[i][j] = A[3 * i + j];
    for (int j = 0; j < 3; ++j) a[i][3 + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0) return false;
    if (piv != col)
      for (int j = 0; j < 6; ++j) std::swap(a[piv][j], a[col][j]);
    double p = a[col][col];
    for (int j = 0; j < 6; ++j) a[col][j] /= p;
    for (int r = 0; r < 3; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      for (int j = 0; j < 6; ++j) a[r][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Ainv[3 * i + j] = a[i][3 + j];
  return true;
}

// [a]x : the matrix with [a]x b = a x b.
void skew(const double* a, double* S) {
  S[0] = 0.0;   S[1] = -a[2]; S[2] = a[1];
  S[3] = a[2];  S[4] = 0.0;   S[5] = -a[0];
  S[6] = -a[1]; S[7] = a[0];  S[8] = 0.0;
}

// Voxel index of one axis: floor(x / r) in binary64.
int64_t axis_key(double x, double r) { return (int64_t)std::floor(x / r); }

// q = R mu + t, evaluated left to right in binary64 (((R0 x + R1 y) + R2 z) + t).
void transform_point(const double* T, const double* mu, double* q) {
  for (int i = 0; i < 3; ++i) {
    double s = T[4 * i + 0] * mu[0];
    s = s + T[4 * i + 1] * mu[1];
    s = s + T[4 * i + 2] * mu[2];
    s = s + T[4 * i + 3];
    q[i] = s;
  }
}

struct VoxelTable {
  std::unordered_map<Key3, int64_t, Key3Hash> index;
  const double* means;  // V x 3
  const double* covs;   // V x 6 (upper triangle)
};

void make_table(const int64_t* vkeys, int64_t V, VoxelTable* tab) {
  tab->index.reserve((size_t)V * 2 + 1);
  for (int64_t v = 0; v < V; ++v)
    tab->index.emplace(Key3{vkeys[3 * v], vkeys[3 * v + 1], vkeys[3 * v + 2]}, v);
}

int64_t lookup(const VoxelTable& tab, const Key3& k) {
  auto it = tab.index.find(k);
  return it == tab.index.end() ? -1 : it->second;
}

// One distribution-to-distribution term (Eq. 3) of source point (mu, C) against
// voxel (mu', C') under pose T, with its Gauss-Newton contributions.
//   d = mu' - (R mu + t)
//   W = (C' + R C R^T)^-1
//   J = d d / d xi = [ R [mu]x , -R ]     (right perturbation, xi = [omega; v])
//   H += J^T W J, b += J^T W d, err += d^T W d
struct Terms {
  double H[36];
  double b[6];
  double err;
  int64_t inliers;
  void clear() { std::memset(this, 0, sizeof(*this)); }
  void add(const Terms& o) {
    for (int i = 0; i < 36; ++i) H[i] += o.H[i];
    for (int i = 0; i < 6; ++i) b[i] += o.b[i];
    err += o.err;
    inliers += o.inliers;
  }
};

void d2d_term(const double* T, const double* mu, const double* C, const double* vmu,
              const double* vC, Terms* acc, double* W_out, double* d_out) {
  double R[9], Rt[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[3 * i + j] = T[4 * i + j];
  mat3_transpose(R, Rt);

  double q[3];
  transform_point(T, mu, q);
  double d[3] = {vmu[0] - q[0], vmu[1] - q[1], vmu[2] - q[2]};

  double RC[9], RCRt[9], M[9], W[9];
  mat3_mul(R, C, RC);
  mat3_mul(RC, Rt, RCRt);
  for (int i = 0; i < 9; ++i) M[i] = vC[i] + RCRt[i];
  if (!mat3_inverse(M, W)) return;  // singular fused covariance: no term

  // J (3x6) = [ R [mu]x , -R ]
  double S[9], RS[9];
  skew(mu, S);
  mat3_mul(R, S, RS);
  double J[18];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      J[6 * i + j] = RS[3 * i + j];
      J[6 * i + 3 + j] = -R[3 * i + j];
    }

  // WJ (3x6), Wd (3)
  double WJ[18], Wd[3];
  for (int i = 0; i < 3; ++i) {
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += W[3 * i + k] * J[6 * k + c];
      WJ[6 * i + c] = s;
    }
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += W[3 * i + k] * d[k];
    Wd[i] = s;
  }
  for (int r = 0; r < 6; ++r) {
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += J[6 * k + r] * WJ[6 * k + c];
      acc->H[6 * r + c] += s;
    }
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += J[6 * k + r] * Wd[k];
    acc->b[r] += s;
  }
  double e = 0.0;
  for (int k = 0; k < 3; ++k) e += d[k] * Wd[k];
  acc->err += e;
  acc->inliers += 1;
  if (W_out) std::memcpy(W_out, W, sizeof(W));
  if (d_out) std::memcpy(d_out, d, sizeof(d));
}

int num_threads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

// Jacobi eigen-decomposition of a symmetric 3x3 matrix (cyclic sweeps of plane
// rotations, Golub & Van Loan Sec. 8.5).  On return w holds the eigenvalues and
// the columns of V the eigenvectors (A = V diag(w) V^T).
void jacobi_eigen3(const double* Ain, double* w, double* V) {
  double A[9];
  std::memcpy(A, Ain, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off == 0.0) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        double apq = A[3 * p + q];
        if (apq == 0.0) continue;
        double app = A[3 * p + p], aqq = A[3 * q + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        // A <- G^T A G with G the rotation in the (p, q) plane.
        for (int k = 0; k < 3; ++k) {
          double akp = A[3 * k + p], akq = A[3 * k + q];
          A[3 * k + p] = c * akp - s * akq;
          A[3 * k + q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = A[3 * p + k], aqk = A[3 * q + k];
          A[3 * p + k] = c * apk - s * aqk;
          A[3 * q + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = V[3 * k + p], vkq = V[3 * k + q];
          V[3 * k + p] = c * vkp - s * vkq;
          V[3 * k + q] = s * vkp + c * vkq;
        }
      }
  }
  w[0] = A[0]; w[1] = A[4]; w[2] = A[8];
}

}  // namespace

extern "C" {

// Per-point voxel keys of a float cloud (n x 3), floor(x / r) per axis.
void oracle_voxel_keys(const float* pts, int64_t n, double r, int64_t* keys) {
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) keys[3 * i + a] = axis_key((double)pts[3 * i + a], r);
}

// Voxel map of a target cloud (Sec. III-A).  Voxels are listed in order of first
// appearance; for each: key (3 x int64), point count N, mean of the point means
// and mean of the point covariances (6 upper-triangular entries), both in
// binary64 with the sum taken in ascending point index and then divided by N.
// Output arrays must hold n entries.  Returns the number of voxels V.
int64_t oracle_build_voxelmap(const float* pts, const float* covs, int64_t n, double r,
                              int64_t* keys, int64_t* counts, double* means, double* vcovs) {
  std::unordered_map<Key3, int64_t, Key3Hash> index;
  index.reserve((size_t)n * 2 + 1);
  std::vector<double> sum_mu, sum_c;
  int64_t V = 0;
  for (int64_t i = 0; i < n; ++i) {
    Key3 k{axis_key((double)pts[3 * i], r), axis_key((double)pts[3 * i + 1], r),
           axis_key((double)pts[3 * i + 2], r)};
    auto it = index.find(k);
    int64_t v;
    if (it == index.end()) {
      v = V++;
      index.emplace(k, v);
      keys[3 * v] = k.x; keys[3 * v + 1] = k.y; keys[3 * v + 2] = k.z;
      counts[v] = 0;
      sum_mu.resize(3 * V, 0.0);
      sum_c.resize(6 * V, 0.0);
    } else {
      v = it->second;
    }
    counts[v] += 1;
    for (int a = 0; a < 3; ++a) sum_mu[3 * v + a] += (double)pts[3 * i + a];
    for (int a = 0; a < 6; ++a) sum_c[6 * v + a] += (double)covs[6 * i + a];
  }
  for (int64_t v = 0; v < V; ++v) {
    double N = (double)counts[v];
    for (int a = 0; a < 3; ++a) means[3 * v + a] = sum_mu[3 * v + a] / N;
    for (int a = 0; a < 6; ++a) vcovs[6 * v + a] = sum_c[6 * v + a] / N;
  }
  return V;
}

// Linearise one VGICP factor (Eqs. 2-3) at T = T_target_source (row-major 4x4).
//   neighbours: 1 (the voxel containing T mu) or 27 (3x3x3 block around it).
//   H (36, row-major), b (6), err (1), inliers (1): outputs.
//   corr (n, may be NULL): voxel index of the point's own voxel, or -1 (1 and 27).
//   qkeys (n x 3, may be NULL): key of T mu.
//   W_out (n x 9), d_out (n x 3) (may be NULL; 1-neighbour mode only): the
//   per-point weight and residual, zero for points without a voxel.
// Sums run over fixed chunks of 4096 points in order, so the result does not
// depend on nthreads.  Returns 0, or -1 for a bad argument.
int oracle_linearize(const int64_t* vkeys, const double* vmeans, const double* vcovs, int64_t V,
                     double r, const float* src, const float* src_covs, int64_t n,
                     const double* T, int neighbours, int nthreads, double* H, double* b,
                     double* err, int64_t* inliers, int64_t* corr, int64_t* qkeys,
                     double* W_out, double* d_out) {
  if (neighbours != 1 && neighbours != 27) return -1;
  if (n < 0 || V < 0 || !(r > 0.0)) return -1;
  VoxelTable tab;
  make_table(vkeys, V, &tab);
  tab.means = vmeans;
  tab.covs = vcovs;

  const int64_t chunk = 4096;
  const int64_t nchunks = (n + chunk - 1) / chunk;
  std::vector<Terms> part((size_t)std::max<int64_t>(nchunks, 1));
  for (auto& p : part) p.clear();

  int nt = num_threads_or_default(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t c = 0; c < nchunks; ++c) {
    Terms acc;
    acc.clear();
    for (int64_t i = c * chunk; i < std::min(n, (c + 1) * chunk); ++i) {
      double mu[3] = {src[3 * i], src[3 * i + 1], src[3 * i + 2]};
      double C[9];
      sym_from_upper(src_covs + 6 * i, C);
      double q[3];
      transform_point(T, mu, q);
      Key3 k{axis_key(q[0], r), axis_key(q[1], r), axis_key(q[2], r)};
      if (qkeys) { qkeys[3 * i] = k.x; qkeys[3 * i + 1] = k.y; qkeys[3 * i + 2] = k.z; }
      int64_t own = lookup(tab, k);
      if (corr) corr[i] = own;
      if (W_out) std::memset(W_out + 9 * i, 0, 9 * sizeof(double));
      if (d_out) std::memset(d_out + 3 * i, 0, 3 * sizeof(double));
      if (neighbours == 1) {
        if (own < 0) continue;
        double vC[9];
        sym_from_upper_d(vcovs + 6 * own, vC);
        d2d_term(T, mu, C, vmeans + 3 * own, vC, &acc, W_out ? W_out + 9 * i : nullptr,
                 d_out ? d_out + 3 * i : nullptr);
      } else {
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int64_t v = lookup(tab, Key3{k.x + dx, k.y + dy, k.z + dz});
              if (v < 0) continue;
              double vC[9];
              sym_from_upper_d(vcovs + 6 * v, vC);
              d2d_term(T, mu, C, vmeans + 3 * v, vC, &acc, nullptr, nullptr);
            }
      }
    }
    part[(size_t)c] = acc;
  }
  Terms tot;
  tot.clear();
  for (int64_t c = 0; c < nchunks; ++c) tot.add(part[(size_t)c]);
  std::memcpy(H, tot.H, sizeof(tot.H));
  std::memcpy(b, tot.b, sizeof(tot.b));
  *err = tot.err;
  *inliers = tot.inliers;
  return 0;
}

// Cost of Eq. 2 at pose T with the correspondences held fixed (corr[i] = voxel
// index or -1).  If W_fixed (n x 9) is given, those weights are used; otherwise W
// is recomputed at T.  Used by finite-difference checks of b and of the exact
// gradient.
double oracle_cost_fixed(const double* vmeans, const double* vcovs, const float* src,
                         const float* src_covs, int64_t n, const double* T, const int64_t* corr,
                         const double* W_fixed) {
  double R[9], Rt[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[3 * i + j] = T[4 * i + j];
  mat3_transpose(R, Rt);
  double total = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = corr[i];
    if (v < 0) continue;
    double mu[3] = {src[3 * i], src[3 * i + 1], src[3 * i + 2]};
    double q[3];
    transform_point(T, mu, q);
    double d[3] = {vmeans[3 * v] - q[0], vmeans[3 * v + 1] - q[1], vmeans[3 * v + 2] - q[2]};
    double W[9];
    if (W_fixed) {
      std::memcpy(W, W_fixed + 9 * i, sizeof(W));
    } else {
      double C[9], vC[9], RC[9], RCRt[9], M[9];
      sym_from_upper(src_covs + 6 * i, C);
      sym_from_upper_d(vcovs + 6 * v, vC);
      mat3_mul(R, C, RC);
      mat3_mul(RC, Rt, RCRt);
      for (int k = 0; k < 9; ++k) M[k] = vC[k] + RCRt[k];
      if (!mat3_inverse(M, W)) continue;
    }
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) total += d[a] * W[3 * a + c] * d[c];
  }
  return total;
}

// Exact gradient of Eq. 2 with respect to the right perturbation xi = [omega; v]
// at T, correspondences fixed, including the change of W with the rotation:
//   g = sum 2 J^T W d  +  [ -u^T dM/domega_i u ]_{i=0..2}  (0 for v),
//   u = W d,  dM/domega_i = R ([e_i]x C - C [e_i]x) R^T.
void oracle_exact_gradient(const double* vmeans, const double* vcovs, const float* src,
                           const float* src_covs, int64_t n, const double* T,
                           const int64_t* corr, double* g) {
  double R[9], Rt[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[3 * i + j] = T[4 * i + j];
  mat3_transpose(R, Rt);
  for (int i = 0; i < 6; ++i) g[i] = 0.0;
  for (int64_t p = 0; p < n; ++p) {
    int64_t v = corr[p];
    if (v < 0) continue;
    double mu[3] = {src[3 * p], src[3 * p + 1], src[3 * p + 2]};
    double C[9], vC[9];
    sym_from_upper(src_covs + 6 * p, C);
    sym_from_upper_d(vcovs + 6 * v, vC);
    Terms t;
    t.clear();
    double W[9], d[3];
    d2d_term(T, mu, C, vmeans + 3 * v, vC, &t, W, d);
    if (t.inliers == 0) continue;
    for (int i = 0; i < 6; ++i) g[i] += 2.0 * t.b[i];
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = W[3 * a] * d[0] + W[3 * a + 1] * d[1] + W[3 * a + 2] * d[2];
    for (int i = 0; i < 3; ++i) {
      double e[3] = {0, 0, 0};
      e[i] = 1.0;
      double E[9], EC[9], CE[9], D[9], RD[9], dM[9];
      skew(e, E);
      mat3_mul(E, C, EC);
      mat3_mul(C, E, CE);
      for (int k = 0; k < 9; ++k) D[k] = EC[k] - CE[k];
      mat3_mul(R, D, RD);
      mat3_mul(RD, Rt, dM);
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) s += u[a] * dM[3 * a + c] * u[c];
      g[i] -= s;
    }
  }
}

// k nearest neighbours (the point itself included) by brute force: neighbours
// ordered by (squared distance, index).  nbr: n x k.
void oracle_knn_bruteforce(const float* pts, int64_t n, int k, int64_t* nbr) {
  std::vector<std::pair<double, int64_t>> cand((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      double dx = (double)pts[3 * j] - pts[3 * i], dy = (double)pts[3 * j + 1] - pts[3 * i + 1],
             dz = (double)pts[3 * j + 2] - pts[3 * i + 2];
      cand[(size_t)j] = {dx * dx + dy * dy + dz * dz, j};
    }
    std::partial_sort(cand.begin(), cand.begin() + std::min<int64_t>(k, n), cand.end());
    for (int a = 0; a < k; ++a) nbr[(int64_t)k * i + a] = a < n ? cand[(size_t)a].second : -1;
  }
}

// Same result as oracle_knn_bruteforce, using a uniform grid of cell size h and
// searching rings of cells until the k-th best distance cannot improve.
void oracle_knn_grid(const float* pts, int64_t n, int k, double h, int nthreads, int64_t* nbr) {
  std::unordered_map<Key3, std::vector<int64_t>, Key3Hash> grid;
  grid.reserve((size_t)n);
  for (int64_t i = 0; i < n; ++i)
    grid[Key3{axis_key(pts[3 * i], h), axis_key(pts[3 * i + 1], h), axis_key(pts[3 * i + 2], h)}]
        .push_back(i);
  int nt = num_threads_or_default(nthreads);
  (void)nt;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nt)
  for (int64_t i = 0; i < n; ++i) {
    double px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    Key3 c{axis_key(px, h), axis_key(py, h), axis_key(pz, h)};
    std::vector<std::pair<double, int64_t>> best;
    for (int64_t s = 0;; ++s) {
      // visit the cells at Chebyshev distance exactly s from c
      for (int64_t dz = -s; dz <= s; ++dz)
        for (int64_t dy = -s; dy <= s; ++dy)
          for (int64_t dx = -s; dx <= s; ++dx) {
            if (std::max({std::llabs(dx), std::llabs(dy), std::llabs(dz)}) != s) continue;
            auto it = grid.find(Key3{c.x + dx, c.y + dy, c.z + dz});
            if (it == grid.end()) continue;
            for (int64_t j : it->second) {
              double ex = (double)pts[3 * j] - px, ey = (double)pts[3 * j + 1] - py,
                     ez = (double)pts[3 * j + 2] - pz;
              best.push_back({ex * ex + ey * ey + ez * ez, j});
            }
          }
      std::sort(best.begin(), best.end());
      if ((int64_t)best.size() > k) best.resize((size_t)k);
      // any point in ring s+1 or beyond is at least s*h away; stop only when
      // the k-th distance is strictly inside that radius, so index tie-breaks hold
      double reach = (double)s * h;
      if ((int64_t)best.size() >= std::min<int64_t>(k, n) &&
          (best.empty() || best.back().first < reach * reach))
        break;
      if ((int64_t)best.size() >= n) break;
    }
    for (int a = 0; a < k; ++a) nbr[(int64_t)k * i + a] = a < (int)best.size() ? best[(size_t)a].second : -1;
  }
}

// Point covariances from given neighbour lists (Sec. III-C/III-D; GICP-style
// regularisation): the sample covariance of the k neighbours (1/k, about their
// centroid) is eigen-decomposed and its eigenvalues, sorted in decreasing order,
// are replaced by (1, 1, eps).  covs: n x 6 upper triangle.
void oracle_regularized_covariances(const float* pts, int64_t n, int k, const int64_t* nbr,
                                    double eps, double* covs) {
  for (int64_t i = 0; i < n; ++i) {
    double m[3] = {0, 0, 0};
    int cnt = 0;
    for (int a = 0; a < k; ++a) {
      int64_t j = nbr[(int64_t)k * i + a];
      if (j < 0) continue;
      for (int c = 0; c < 3; ++c) m[c] += pts[3 * j + c];
      ++cnt;
    }
    for (int c = 0; c < 3; ++c) m[c] /= cnt;
    double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < k; ++a) {
      int64_t j = nbr[(int64_t)k * i + a];
      if (j < 0) continue;
      double e[3] = {pts[3 * j] - m[0], pts[3 * j + 1] - m[1], pts[3 * j + 2] - m[2]};
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) S[3 * r + c] += e[r] * e[c];
    }
    for (int c = 0; c < 9; ++c) S[c] /= cnt;
    double w[3], V[9];
    jacobi_eigen3(S, w, V);
    int order[3] = {0, 1, 2};
    std::sort(order, order + 3, [&](int a, int c) { return w[a] > w[c]; });
    double lam[3] = {1.0, 1.0, eps};
    double Cr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 3; ++a) {
      int col = order[a];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Cr[3 * r + c] += lam[a] * V[3 * r + col] * V[3 * c + col];
    }
    covs[6 * i + 0] = Cr[0]; covs[6 * i + 1] = Cr[1]; covs[6 * i + 2] = Cr[2];
    covs[6 * i + 3] = Cr[4]; covs[6 * i + 4] = Cr[5]; covs[6 * i + 5] = Cr[8];
  }
}

// Voxel-grid downsampling with timestamp averaging (Sec. III-C).  Points are
// taken in index order.  A point's voxel is floor(p / r); the voxel's reference
// time is that of its first point; a point whose time differs from it by more
// than `split` (the paper's example: a tenth of the scan duration) goes to the
// voxel's second, separate output voxel, so that the first and last points of a
// scan are not fused.  Output voxels are numbered in order of first appearance;
// each holds the binary64 mean of its points' positions and times (sums in
// index order, then / N), rounded to float32.  times == NULL or split <= 0: no
// split, no times.  Returns the number of output voxels.
int64_t oracle_downsample(const float* pts, const float* times, int64_t n, double r, double split,
                          float* out_pts, float* out_times, int64_t* out_counts) {
  struct First {
    int64_t index;
    double time;
  };
  std::unordered_map<Key3, First, Key3Hash> first;
  std::map<std::pair<Key3, int>, int64_t> id;
  std::vector<double> sum;  // 4 per output voxel: x, y, z, t
  std::vector<int64_t> cnt;
  const bool timed = times != nullptr && split > 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const Key3 k{axis_key(pts[3 * i], r), axis_key(pts[3 * i + 1], r), axis_key(pts[3 * i + 2], r)};
    const double ti = times ? (double)times[i] : 0.0;
    auto f = first.find(k);
    if (f == first.end()) f = first.emplace(k, First{i, ti}).first;
    const int sub = timed && std::fabs(ti - f->second.time) > split ? 1 : 0;
    auto g = id.find({k, sub});
    if (g == id.end()) {
      g = id.emplace(std::make_pair(k, sub), (int64_t)cnt.size()).first;
      cnt.push_back(0);
      sum.insert(sum.end(), {0.0, 0.0, 0.0, 0.0});
    }
    const int64_t v = g->second;
    for (int c = 0; c < 3; ++c) sum[4 * v + c] += pts[3 * i + c];
    sum[4 * v + 3] += ti;
    ++cnt[v];
  }
  const int64_t V = (int64_t)cnt.size();
  for (int64_t v = 0; v < V; ++v) {
    for (int c = 0; c < 3; ++c) out_pts[3 * v + c] = (float)(sum[4 * v + c] / (double)cnt[v]);
    if (out_times) out_times[v] = (float)(sum[4 * v + 3] / (double)cnt[v]);
    out_counts[v] = cnt[v];
  }
  return V;
}

// Eigen-decomposition exposed for its own pin (against a library routine).
void oracle_jacobi_eigen3(const double* A, double* w, double* V) { jacobi_eigen3(A, w, V); }

// 3x3 inverse exposed for its own pin.
int oracle_mat3_inverse(const double* A, double* Ainv) { return mat3_inverse(A, Ainv) ? 0 : -1; }

}  // extern "C"
