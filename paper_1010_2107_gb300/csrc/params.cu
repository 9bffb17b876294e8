// params.cu -- host-side derivation of the constants the device integrands
// read (slot layout in integrands.cuh) and of the scale that turns their
// dimensionless values into the integrand's units.
#include <algorithm>
#include <cmath>
#include <string>

#include "integrands.cuh"
#include "kernels.h"

namespace gv {

int expected_nparams(int kind, int d) {
  switch (kind) {
    case VG_GENZ_GAUSSIAN:
    case VG_GENZ_PRODUCT_PEAK: return 2 * d;
    case VG_GENZ_CORNER_PEAK: return d;
    case VG_GENZ_OSCILLATORY: return d + 1;
    case VG_DOUBLE_GAUSSIAN: return 3;
    case VG_RAMBO_BW: return VG_RB_NPARAMS;
    case VG_GENZ_CONTINUOUS: return 2 * d;
    case VG_GENZ_DISCONTINUOUS: return d + (d < 2 ? d : 2);
    case VG_W_MUNU: return VG_W_NPARAMS;
    default: return -1;
  }
}

bool derive_params(int kind, int d, const double* p, double* dv, double* scale, std::string* why) {
  std::fill(dv, dv + gv::kNumDerived, 0.0);
  *scale = 1.0;
  const int M = gv::kMaxDim, S = gv::kScalar;
  switch (kind) {
    case VG_GENZ_GAUSSIAN:
      for (int i = 0; i < d; ++i) {
        dv[i] = p[i] * p[i];
        dv[M + i] = p[d + i];
        dv[2 * M + i] = p[i];
      }
      return true;
    case VG_GENZ_PRODUCT_PEAK:
      for (int i = 0; i < d; ++i) {
        dv[i] = 1.0 / (p[i] * p[i]);
        dv[M + i] = p[d + i];
      }
      return true;
    case VG_GENZ_CORNER_PEAK:
      for (int i = 0; i < d; ++i) dv[i] = p[i];
      dv[S] = -(double)(d + 1);
      return true;
    case VG_GENZ_OSCILLATORY:
      for (int i = 0; i < d; ++i) dv[i] = p[i];
      dv[S] = 2.0 * M_PI * p[d];
      return true;
    case VG_GENZ_CONTINUOUS:
      for (int i = 0; i < d; ++i) {
        dv[i] = p[i];
        dv[M + i] = p[d + i];
      }
      return true;
    case VG_GENZ_DISCONTINUOUS:
      for (int i = 0; i < d; ++i) dv[i] = p[i];
      dv[S] = p[d];
      dv[S + 1] = d > 1 ? p[d + 1] : 2.0;
      return true;
    case VG_DOUBLE_GAUSSIAN: {
      const double w = p[2];
      if (!(w > 0.0)) {
        *why = "double Gaussian width must be positive";
        return false;
      }
      dv[S] = p[0];
      dv[S + 1] = p[1];
      dv[S + 2] = 1.0 / (w * w);
      dv[S + 3] = 0.5 * std::pow(w * std::sqrt(M_PI), -(double)d);
      dv[S + 4] = w;
      return true;
    }
    case VG_RAMBO_BW: {
      const int n = (int)p[VG_RB_N];
      if (n < 2 || 4 * n != d || (double)n != p[VG_RB_N]) {
        *why = "RAMBO needs ndim = 4 n with integer n >= 2";
        return false;
      }
      const double rs = p[VG_RB_SQRTS], s = rs * rs, Mw = p[VG_RB_M], Gw = p[VG_RB_GAMMA];
      if (!(rs > 0.0)) {
        *why = "RAMBO needs sqrt(s) > 0";
        return false;
      }
      const int cut = (int)p[VG_RB_CUT], obs = (int)p[VG_RB_OBS];
      if (cut < 0 || cut > 2 || obs < 0 || obs > 3) {
        *why = "RAMBO cut must be 0..2 and observable 0..3";
        return false;
      }
      if (cut == 1 && !(p[VG_RB_WC] > 0.0)) {
        *why = "sigmoid cut width must be positive";
        return false;
      }
      double V = std::pow(M_PI / 2.0, n - 1) * std::pow(s, n - 2);
      for (int i = 2; i <= n - 1; ++i) V /= i;
      for (int i = 2; i <= n - 2; ++i) V /= i;
      dv[gv::RB_N] = n;
      dv[gv::RB_MU] = Mw * Mw / s;
      dv[gv::RB_MUG] = Mw * Gw / s;
      dv[gv::RB_MUG2] = (Mw * Gw / s) * (Mw * Gw / s);
      dv[gv::RB_PTMIN] = p[VG_RB_PTMIN] / rs;
      dv[gv::RB_DR2] = p[VG_RB_DRMIN] * p[VG_RB_DRMIN];
      dv[gv::RB_CUT] = cut;
      dv[gv::RB_T] = p[VG_RB_T] / rs;
      dv[gv::RB_INVWC] = cut == 1 ? rs / p[VG_RB_WC] : 0.0;
      dv[gv::RB_OBS] = obs;
      dv[gv::RB_DMU_DM] = 2.0 * Mw / s;
      dv[gv::RB_DMUG_DM] = Gw / s;
      dv[gv::RB_DMUG_DG] = Mw / s;
      dv[gv::RB_INVWC_GEV] = cut == 1 ? 1.0 / p[VG_RB_WC] : 0.0;
      // obs 0: V_n * s^-(n+1) (dimensionless product); 1: V_n; 2: V_n s;
      // 3: V_n / s.
      switch (obs) {
        case 0: *scale = V * std::pow(s, -(double)(n + 1)); break;
        case 1: *scale = V; break;
        case 2: *scale = V * s; break;
        default: *scale = V / s; break;
      }
      return true;
    }
    case VG_W_MUNU: {
      if (d != 5) {
        *why = "the W -> mu nu integrand has ndim 5";
        return false;
      }
      const double rs = p[VG_W_SQRTS], S = rs * rs, Mw = p[VG_W_M], Gw = p[VG_W_GAMMA];
      if (!(rs > 0.0 && Mw > 0.0 && Gw > 0.0 && p[VG_W_SMIN] >= 0.0 && p[VG_W_SMIN] < S)) {
        *why = "W -> mu nu needs sqrt(S), M, Gamma > 0 and 0 <= SMIN < S";
        return false;
      }
      if (p[VG_W_CUTS] != 0.0 && p[VG_W_CUTS] != 1.0) {
        *why = "W -> mu nu CUTS must be 0 or 1";
        return false;
      }
      const double rlo = std::atan((p[VG_W_SMIN] - Mw * Mw) / (Mw * Gw));
      const double rhi = std::atan((S - Mw * Mw) / (Mw * Gw));
      const double g2 = 8.0 * Mw * Mw * p[VG_W_GF] / std::sqrt(2.0);
      const double pb = 0.3893793721e9;  // GeV^-2 -> pb
      dv[W_RLO] = rlo;
      dv[W_DRHO] = rhi - rlo;
      dv[W_M2] = Mw * Mw;
      dv[W_MG] = Mw * Gw;
      dv[W_INVS] = 1.0 / S;
      dv[W_PT2] = 4.0 * p[VG_W_PTMIN] * p[VG_W_PTMIN];
      dv[W_ETA] = p[VG_W_ETAMAX];
      dv[W_CUTS] = p[VG_W_CUTS];
      dv[W_K] = p[VG_W_AU] * p[VG_W_AD] * (rhi - rlo) * g2 * g2 * p[VG_W_VUD] * p[VG_W_VUD] * pb /
                (48.0 * M_PI * S * Mw * Gw);
      dv[W_ALU] = p[VG_W_ALU];
      dv[W_BU] = p[VG_W_BU];
      dv[W_ALD] = p[VG_W_ALD];
      dv[W_BD] = p[VG_W_BD];
      return true;
    }
    default:
      *why = "unknown integrand kind";
      return false;
  }
}

}  // namespace gv
