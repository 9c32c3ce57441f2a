// Host binary64 pose algebra for the optimizer side of the factor (arXiv
// 2202.00242 Sec. III-A: the factor is re-linearized at each iteration; the
// perturbation is the right one, T <- T Exp(xi), xi = [omega; v]).
//   Exp        : closed form of the SE(3) matrix exponential (Rodrigues for the
//                rotation, V = I + (1-cos)/th^2 W + (th-sin)/th^3 W^2 for v)
//   J_r(xi)    : right Jacobian, Exp(xi + d) ~ Exp(xi) Exp(J_r(xi) d); for
//                xi = [phi; rho] it is J_l(-xi) with the SE(3) left Jacobian
//                [[J(phi), 0], [Q(rho, phi), J(phi)]] of Barfoot (State
//                Estimation for Robotics, Sec. 7.1.5)
//   solve6     : Cholesky of the 6x6 normal equations (H + lambda diag(H)) x = -b
#include <cmath>
#include <cstring>

#include "vgicp.h"
#include "vgicp_internal.h"

namespace {

void hat3(const double* w, double* W) {
  W[0] = 0.0;   W[1] = -w[2]; W[2] = w[1];
  W[3] = w[2];  W[4] = 0.0;   W[5] = -w[0];
  W[6] = -w[1]; W[7] = w[0];  W[8] = 0.0;
}

void mm3(const double* A, const double* B, double* C) {
  double T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      T[3 * i + j] = s;
    }
  std::memcpy(C, T, sizeof(T));
}

// Coefficients of the SO(3) series with small-angle limits.
void so3_coeffs(double th, double* a, double* b, double* c) {
  // a = sin th / th, b = (1 - cos th) / th^2, c = (th - sin th) / th^3
  if (th < 1e-4) {
    const double t2 = th * th;
    *a = 1.0 - t2 / 6.0;
    *b = 0.5 - t2 / 24.0;
    *c = 1.0 / 6.0 - t2 / 120.0;
  } else {
    *a = std::sin(th) / th;
    *b = (1.0 - std::cos(th)) / (th * th);
    *c = (th - std::sin(th)) / (th * th * th);
  }
}

// SE(3) left Jacobian blocks for xi = [phi; rho]: J (3x3) and Q (3x3).
void left_jacobian(const double* phi, const double* rho, double* J, double* Q) {
  const double th = std::sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
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
    const double s = std::sin(th), co = std::cos(th);
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

}  // namespace

extern "C" {

int vgicp_se3_exp(const double* xi, double* T) {
  if (!xi || !T) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  const double* w = xi;
  const double* v = xi + 3;
  const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
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
  return VGICP_OK;
}

int vgicp_se3_right_jacobian(const double* xi, double* J6) {
  if (!xi || !J6) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
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
  return VGICP_OK;
}

int vgicp_pose_mul(const double* A, const double* B, double* C) {
  if (!A || !B || !C) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  double T[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[4 * i + k] * B[4 * k + j];
      T[4 * i + j] = s;
    }
  std::memcpy(C, T, sizeof(T));
  return VGICP_OK;
}

int vgicp_binary_factor(const double* H, const double* b, const double* T, double* H2,
                        double* b2) {
  if (!H || !b || !T || !H2 || !b2) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  // A = [I, -Ad(T^-1)] maps [delta_i; delta_j] to xi.  With T^-1 = (R^T, -R^T t)
  // and xi = [omega; v]: Ad(T^-1) = [[R^T, 0], [[-R^T t]x R^T, R^T]].
  double Rt[9], ti[3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Rt[3 * r + c] = T[4 * c + r];
  for (int r = 0; r < 3; ++r)
    ti[r] = -(Rt[3 * r] * T[3] + Rt[3 * r + 1] * T[7] + Rt[3 * r + 2] * T[11]);
  double TX[9], TXR[9];
  hat3(ti, TX);
  mm3(TX, Rt, TXR);
  double A[6 * 12] = {0};
  for (int r = 0; r < 6; ++r) A[12 * r + r] = 1.0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      A[12 * r + 6 + c] = -Rt[3 * r + c];            // omega <- omega_j
      A[12 * (3 + r) + 9 + c] = -Rt[3 * r + c];      // v <- v_j
      A[12 * (3 + r) + 6 + c] = -TXR[3 * r + c];     // v <- omega_j
    }
  double HA[6 * 12];
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 12; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += H[6 * r + k] * A[12 * k + c];
      HA[12 * r + c] = acc;
    }
  for (int r = 0; r < 12; ++r) {
    for (int c = 0; c < 12; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 6; ++k) acc += A[12 * k + r] * HA[12 * k + c];
      H2[12 * r + c] = acc;
    }
    double acc = 0.0;
    for (int k = 0; k < 6; ++k) acc += A[12 * k + r] * b[k];
    b2[r] = acc;
  }
  return VGICP_OK;
}

int vgicp_solve6(const double* H, const double* b, double lambda, double* xi) {
  if (!H || !b || !xi) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  double A[36], L[36] = {0};
  for (int i = 0; i < 36; ++i) A[i] = H[i];
  for (int i = 0; i < 6; ++i) A[7 * i] += lambda * H[7 * i];
  for (int j = 0; j < 6; ++j) {
    double d = A[7 * j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0) || !std::isfinite(d))
      return vgicp::set_error(VGICP_ERR_INVALID_ARG, "H is not positive definite");
    L[7 * j] = std::sqrt(d);
    for (int i = j + 1; i < 6; ++i) {
      double s = A[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = s / L[7 * j];
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = -b[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
    y[i] = s / L[7 * i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * xi[k];
    xi[i] = s / L[7 * i];
  }
  return VGICP_OK;
}

}  // extern "C"
