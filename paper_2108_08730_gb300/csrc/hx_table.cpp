// Weight-table fit of the adaptive stencil (Section 2.2), host FP64.
//
// Unknowns, node-major as in the paper: w = [w^(0); w^(1); ...], each
// w^(i) = [ws1, ws2, wm1, wm2, wm3] at 1/G_i = i * d_inv_g.  Rows:
//   data rows   H^(i) w^(i) = g^(i)              (one per plane-wave direction)
//   smooth rows sqrt(lambda) (w_l^(i+1) - w_l^(i)) = 0   for l = 0..4
// Ordered node by node, every row touches only the 10 columns of nodes i and
// i+1, so the triangular factor R of a Givens QR stays inside a band of width
// 10.  Rows are rotated into R one at a time (numerically orthogonal, no
// normal equations), then R w = Q^T b is back-substituted.
#include <cmath>
#include <cstring>
#include <vector>

#include "hx_internal.h"

namespace hx {

namespace {

constexpr int kW = 10;  // band width of R: columns j .. j+9

struct BandQR {
  int n;
  std::vector<double> R;     // n x kW, R[j*kW + k] = R(j, j+k)
  std::vector<double> qtb;   // n
  std::vector<char> filled;  // R row j has been set

  explicit BandQR(int n_) : n(n_), R((size_t)n_ * kW, 0.0), qtb(n_, 0.0), filled(n_, 0) {}

  // Rotate the row (values on columns c0 .. c0+kW-1, rhs b) into R.
  void add_row(int c0, const double* vals, double b) {
    double row[2 * kW];
    std::memset(row, 0, sizeof(row));
    for (int k = 0; k < kW; ++k) row[k] = vals[k];
    for (int j = c0; j < c0 + kW && j < n; ++j) {
      const int o = j - c0;  // position of column j in `row`
      double x = row[o];
      if (x == 0.0) continue;
      double* Rj = &R[(size_t)j * kW];
      if (!filled[j]) {
        for (int k = 0; k < kW && o + k < 2 * kW; ++k) Rj[k] = row[o + k];
        qtb[j] = b;
        filled[j] = 1;
        return;
      }
      const double r = Rj[0];
      const double rho = std::hypot(r, x);
      const double c = r / rho, s = x / rho;
      for (int k = 0; k < kW && o + k < 2 * kW; ++k) {
        const double rk = Rj[k], xk = row[o + k];
        Rj[k] = c * rk + s * xk;
        row[o + k] = -s * rk + c * xk;
      }
      const double t = qtb[j];
      qtb[j] = c * t + s * b;
      b = -s * t + c * b;
    }
  }

  bool solve(std::vector<double>& w) const {
    w.assign(n, 0.0);
    for (int j = n - 1; j >= 0; --j) {
      const double* Rj = &R[(size_t)j * kW];
      if (!filled[j] || Rj[0] == 0.0 || !std::isfinite(Rj[0])) return false;
      double acc = qtb[j];
      for (int k = 1; k < kW && j + k < n; ++k) acc -= Rj[k] * w[j + k];
      w[j] = acc / Rj[0];
    }
    return true;
  }
};

// One data row of Eq. linear_basic at 1/G = inv_g for the unit direction
// (cos(phi)cos(theta), cos(phi)sin(theta), sin(phi)).
void linear_row(double inv_g, double theta, double phi, double H[5], double* g) {
  const double two_pi = 2.0 * M_PI;
  const double ca = std::cos(two_pi * std::cos(phi) * std::cos(theta) * inv_g);
  const double cb = std::cos(two_pi * std::cos(phi) * std::sin(theta) * inv_g);
  const double cc = std::cos(two_pi * std::sin(phi) * inv_g);
  const double A = ca * cb * cc;
  const double B = ca * cb + ca * cc + cb * cc;
  const double C = ca + cb + cc;
  const double K = 2.0 * M_PI * M_PI * inv_g * inv_g;
  H[0] = 0.5 * (3.0 + 3.0 * A - B - C);
  H[1] = 0.5 * (1.0 + 3.0 * A - (5.0 / 3.0) * B + (1.0 / 3.0) * C);
  H[2] = K * (A - 1.0);
  H[3] = K * (6.0 * A - 2.0 * C);
  H[4] = K * (12.0 * A - 4.0 * B);
  *g = 0.5 * ((2.0 * K + 3.0) * A - B + C - 3.0);
}

}  // namespace

int build_weight_table(const double* theta_deg, int n_theta, const double* phi_deg, int n_phi,
                       double inv_g_max, double d_inv_g, double lambda, double* out, int capacity,
                       int* n_g_out, std::string* err) {
  if (!theta_deg || !phi_deg || n_theta < 1 || n_phi < 1) {
    *err = "angle lists must be non-empty";
    return HX_ERR_ARG;
  }
  if (!(d_inv_g > 0.0) || !(inv_g_max > d_inv_g) || !(lambda > 0.0) || !std::isfinite(lambda)) {
    *err = "need 0 < d_inv_g < inv_g_max and lambda > 0";
    return HX_ERR_ARG;
  }
  const int n_g = (int)std::lround(inv_g_max / d_inv_g) + 1;
  if (n_g_out) *n_g_out = n_g;
  if (n_g > 1000000) {
    *err = "table too large";
    return HX_ERR_ARG;
  }
  if (!out || capacity < 7 * n_g) {
    *err = "table_out capacity must be >= 7 * n_g";
    return HX_ERR_ARG;
  }
  const int n = 5 * n_g;
  BandQR qr(n);
  const double sl = std::sqrt(lambda);
  double vals[kW];
  for (int i = 0; i < n_g; ++i) {
    const double inv_g = i * d_inv_g;
    for (int p = 0; p < n_phi; ++p) {
      for (int t = 0; t < n_theta; ++t) {
        double H[5], g;
        linear_row(inv_g, theta_deg[t] * M_PI / 180.0, phi_deg[p] * M_PI / 180.0, H, &g);
        for (int k = 0; k < kW; ++k) vals[k] = k < 5 ? H[k] : 0.0;
        qr.add_row(5 * i, vals, g);
      }
    }
    if (i + 1 < n_g) {
      for (int l = 0; l < 5; ++l) {
        for (int k = 0; k < kW; ++k) vals[k] = 0.0;
        vals[l] = -sl;
        vals[5 + l] = sl;
        qr.add_row(5 * i, vals, 0.0);
      }
    }
  }
  std::vector<double> w;
  if (!qr.solve(w)) {
    *err = "weight fit is rank deficient";
    return HX_ERR_NUMERIC;
  }
  for (int i = 0; i < n_g; ++i) {
    const double ws1 = w[5 * i], ws2 = w[5 * i + 1];
    const double wm1 = w[5 * i + 2], wm2 = w[5 * i + 3], wm3 = w[5 * i + 4];
    double* o = out + 7 * (size_t)i;
    o[0] = ws1;
    o[1] = ws2;
    o[2] = 1.0 - ws1 - ws2;                                  // Eq. eqsws
    o[3] = wm1;
    o[4] = wm2;
    o[5] = wm3;
    o[6] = (1.0 - wm1 - 6.0 * wm2 - 12.0 * wm3) / 8.0;       // Eq. eqswm, per point
  }
  return HX_OK;
}

}  // namespace hx
