// Binary64 SE(3) algebra of the factor's pose variable (arXiv 2202.00242
// Sec. III-A: the factor is re-linearized at each optimizer iteration; the
// perturbation is the right one, T <- T Exp(xi), xi = [omega; v]).  The same
// inline functions serve the host pose API and the device-side pose composition
// of differentiable plan evaluations (one formula, evaluated in binary64 on
// either side; contraction into FMAs may differ in the last bits).
//   exp            : closed form of the SE(3) matrix exponential (Rodrigues for
//                    the rotation, V = I + (1-cos)/th^2 W + (th-sin)/th^3 W^2)
//   right_jacobian : J_r(xi) with Exp(xi + d) ~ Exp(xi) Exp(J_r(xi) d); for
//                    xi = [phi; rho] it is J_l(-xi) with the SE(3) left Jacobian
//                    [[J(phi), 0], [Q(rho, phi), J(phi)]] of Barfoot (State
//                    Estimation for Robotics, Sec. 7.1.5)
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "vgicp_device.cuh"

#ifdef __CUDACC__
#define VGICP_HD __host__ __device__ __forceinline__
#else
#define VGICP_HD inline
#endif

namespace vgicp {
namespace se3 {

VGICP_HD void hat3(const double* w, double* W) {
  W[0] = 0.0;   W[1] = -w[2]; W[2] = w[1];
  W[3] = w[2];  W[4] = 0.0;   W[5] = -w[0];
  W[6] = -w[1]; W[7] = w[0];  W[8] = 0.0;
}

VGICP_HD void mm3(const double* A, const double* B, double* C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      T[3 * i + j] = s;
    }
  for (int i = 0; i < 9; ++i) C[i] = T[i];
}

// Coefficients of the SO(3) series with small-angle limits:
// a = sin th / th, b = (1 - cos th) / th^2, c = (th - sin th) / th^3.
VGICP_HD void so3_coeffs(double th, double* a, double* b, double* c) {
  if (th < 1e-4) {
    const double t2 = th * th;
    *a = 1.0 - t2 / 6.0;
    *b = 0.5 - t2 / 24.0;
    *c = 1.0 / 6.0 - t2 / 120.0;
  } else {
    *a = sin(th) / th;
    *b = (1.0 - cos(th)) / (th * th);
    *c = (th - sin(th)) / (th * th * th);
  }
}

// SE(3) left Jacobian blocks for xi = [phi; rho]: J (3x3) and Q (3x3).
VGICP_HD void left_jacobian(const double* phi, const double* rho, double* J, double* Q) {
  const double th = sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  double a, b, c;
  so3_coeffs(th, &a, &b, &c);
  double P[9], P2[9], Rh[9];
  hat3(phi, P);
  mm3(P, P, P2);
  hat3(rho, Rh);
  for (int i = 0; i < 9; ++i) J[i] = (i % 4 == 0 ? 1.0 : 0.0) + b * P[i] + c * P2[i];
  // Q = 1/2 Rh + c1 (P Rh + Rh P + P Rh P) + c2 (P P Rh + Rh P P - 3 P Rh P)
  //       + c3 (P Rh P P + P P Rh P)
  double c1, c2, c3;
  if (th < 1e-3) {
    const double t2 = th * th;
    // Taylor series of the three coefficients below
    c1 = 1.0 / 6.0 - t2 / 120.0;
    c2 = 1.0 / 24.0 - t2 / 720.0;
    c3 = 1.0 / 120.0 - t2 / 2520.0;
  } else {
    const double s = sin(th), co = cos(th);
    c1 = (th - s) / (th * th * th);
    c2 = (th * th + 2.0 * co - 2.0) / (2.0 * th * th * th * th);
    c3 = (2.0 * th - 3.0 * s + th * co) / (2.0 * th * th * th * th * th);
  }
  double PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
  mm3(P, Rh, PR);
  mm3(Rh, P, RP);
  mm3(PR, P, PRP);
  mm3(P, PR, PPR);
  mm3(RP, P, RPP);
  mm3(PRP, P, PRPP);
  mm3(P, PRP, PPRP);
  for (int i = 0; i < 9; ++i)
    Q[i] = 0.5 * Rh[i] + c1 * (PR[i] + RP[i] + PRP[i]) + c2 * (PPR[i] + RPP[i] - 3.0 * PRP[i]) +
           c3 * (PRPP[i] + PPRP[i]);
}

// T (row-major 4x4) = Exp(xi), xi = [omega; v].
VGICP_HD void expmap(const double* xi, double* T) {
  const double* w = xi;
  const double* v = xi + 3;
  const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  double a, b, c;
  so3_coeffs(th, &a, &b, &c);
  double W[9], W2[9];
  hat3(w, W);
  mm3(W, W, W2);
  double R[9], V[9];
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    R[i] = I + a * W[i] + b * W2[i];
    V[i] = I + b * W[i] + c * W2[i];
  }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) T[4 * i + j] = R[3 * i + j];
    T[4 * i + 3] = V[3 * i] * v[0] + V[3 * i + 1] * v[1] + V[3 * i + 2] * v[2];
  }
  T[12] = T[13] = T[14] = 0.0;
  T[15] = 1.0;
}

// J (row-major 6x6) with Exp(xi + d) = Exp(xi) Exp(J d) + O(|d|^2).
VGICP_HD void right_jacobian(const double* xi, double* J6) {
  const double phi[3] = {-xi[0], -xi[1], -xi[2]};
  const double rho[3] = {-xi[3], -xi[4], -xi[5]};
  double J[9], Q[9];
  left_jacobian(phi, rho, J, Q);
  for (int i = 0; i < 36; ++i) J6[i] = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      J6[6 * i + j] = J[3 * i + j];            // omega <- omega
      J6[6 * (3 + i) + 3 + j] = J[3 * i + j];  // v <- v
      J6[6 * (3 + i) + j] = Q[3 * i + j];      // v <- omega
    }
}

// C = A B (4x4, row-major; C may alias A or B).
VGICP_HD void pose_mul(const double* A, const double* B, double* C) {
  double T[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
      T[4 * i + j] = s;
    }
  for (int i = 0; i < 16; ++i) C[i] = T[i];
}

// A finite rigid transform: finite entries, last row 0 0 0 1, R^T R = I within
// 1e-5 and det R > 0.
VGICP_HD bool rigid(const double* T) {
  for (int i = 0; i < 16; ++i)
    if (!isfinite(T[i])) return false;
  if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0) return false;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += T[4 * k + i] * T[4 * k + j];
      if (fabs(s - (i == j ? 1.0 : 0.0)) > 1e-5) return false;
    }
  const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                     T[2] * (T[4] * T[9] - T[5] * T[8]);
  return det > 0.0;
}

// The factor descriptor of pose T: float32 and binary64 copies of R and t, and
// max |t_i| rounded up to float32 (the bound the exact-key test uses).
VGICP_HD PairDesc pair_desc(const double* T, int32_t map, int32_t src) {
  PairDesc p = {};
  double tmax = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      p.R[3 * i + j] = (float)T[4 * i + j];
      p.R64[3 * i + j] = T[4 * i + j];
    }
    p.t[i] = (float)T[4 * i + 3];
    p.t64[i] = T[4 * i + 3];
    tmax = fmax(tmax, fabs(T[4 * i + 3]));
  }
  float tm = (float)tmax;
  if ((double)tm < tmax) tm = nextafterf(tm, INFINITY);
  p.tmax = tm;
  p.map = map;
  p.src = src;
  return p;
}

}  // namespace se3
}  // namespace vgicp
