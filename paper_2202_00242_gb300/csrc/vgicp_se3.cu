// Host binary64 pose algebra for the optimizer side of the factor (arXiv
// 2202.00242 Sec. III-A: the factor is re-linearized at each iteration; the
// perturbation is the right one, T <- T Exp(xi), xi = [omega; v]).  Exp, the
// right Jacobian and the pose product are the inline functions of
// vgicp_se3.cuh, shared with the device-side pose composition.
//   solve6     : Cholesky of the 6x6 normal equations (H + lambda diag(H)) x = -b
#include <cmath>
#include <cstring>

#include "vgicp.h"
#include "vgicp_internal.h"
#include "vgicp_se3.cuh"

using vgicp::se3::hat3;
using vgicp::se3::mm3;

extern "C" {

int vgicp_se3_exp(const double* xi, double* T) {
  if (!xi || !T) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  vgicp::se3::expmap(xi, T);
  return VGICP_OK;
}

int vgicp_se3_right_jacobian(const double* xi, double* J6) {
  if (!xi || !J6) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  vgicp::se3::right_jacobian(xi, J6);
  return VGICP_OK;
}

int vgicp_pose_mul(const double* A, const double* B, double* C) {
  if (!A || !B || !C) return vgicp::set_error(VGICP_ERR_INVALID_ARG, "null argument");
  vgicp::se3::pose_mul(A, B, C);
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
