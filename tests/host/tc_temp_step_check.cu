// Host program that checks temp_blocks_step (the temperature blocks stepped from T to
// T + dT to first order, used for the forward-difference Jacobian's temperature column)
// against chem_T and cool_T evaluated at T + dT (not part of libtc_gb300.so; built and
// run by tests/test_temp_step.py with the library's csrc/ on the include path).
//
// Usage: tc_temp_step_check IN
//   IN: n as int64, then 12 arrays of n doubles (n, chi_pe, chi_lw, f_shld_H2, f_shld_C,
//       F_LyC, xi, Z'_g, Z'_d, T, x_H2, x_H+), then dt as a double (unused).
// For every cell, at its own T and at eleven temperatures from 12 K to 1e7 K, and with
// every physics switch off and on, each field's change is compared:
//   exact  d_e = f(T + dT) - f(T)    (chem_T / cool_T at T + dT, dT = 1e-7 T)
//   step   d_s = step(T + dT) - f(T)
// A first-order step differs from the exact change by its second-order term, about
// |g| / 2 of it where g = d_e / f is the field's relative change, so the normalised
// error |d_s - d_e| / ((|g| + 1e-5) |d_e| + 1e-12 |f|) (the last term for the curvature
// near a stationary point of the factor, and rounding) stays below 1 for a correct step;
// a wrong coefficient or sign makes it of order 1 / |g|, or |g| / 1e-12.  Changes below
// 1e-11 |f| are checked in absolute terms instead: |d_s - d_e| must stay below 1e-10 |f|.
// Prints one JSON object: the largest normalised error per field.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "tc_phys.cuh"

using namespace tcg;

namespace {
constexpr int NCHEM = sizeof(ChemT<double>) / sizeof(double);
constexpr int NCOOL = sizeof(CoolT<double>) / sizeof(double);
static_assert(NCHEM * sizeof(double) == sizeof(ChemT<double>), "ChemT holds doubles only");
static_assert(NCOOL * sizeof(double) == sizeof(CoolT<double>), "CoolT holds doubles only");
const char* kChemNames[NCHEM] = {"T",    "lnT",   "sqT",   "invT",  "S",     "kgr",   "arr",   "kci",   "kcdH",
                                 "kcdH2", "arrC", "kCpH2", "xMH_T", "xe_hot", "wdH3T", "wdHex", "wdC3T", "wdCex"};
const char* kCoolNames[NCOOL] = {"fcA",  "fcB",  "eps_num", "lyaE", "ffrr",   "cpke",   "cpkH", "cpb", "ok10",
                                 "ob1",  "ob2",  "ob21",    "ck10", "cb1",    "cb2",    "cb21", "rvLlow",
                                 "rvLLTE", "coA", "coN",    "grT",  "grB",    "nebT",   "nebX", "cie"};
static_assert(sizeof(kChemNames) / sizeof(kChemNames[0]) == NCHEM, "one name per ChemT field");
static_assert(sizeof(kCoolNames) / sizeof(kCoolNames[0]) == NCOOL, "one name per CoolT field");

// normalised error of one field (see the header); NaN stays NaN
double field_err(double f, double exact, double step) {
  if (std::fabs(f) < 1e-290) return 0.0;  // underflowed factors (zero or subnormal)
  const double de = exact - f, ds = step - f;
  if (!(std::fabs(de) > 1e-11 * std::fabs(f))) {
    const double a = std::fabs(ds - de) / (1e-10 * std::fabs(f));
    return (a == a) ? a : 1e300;
  }
  // second-order term ~|g| |d_e| / 2; near a stationary point of the factor (d_e ~ 0) the
  // curvature term, ~(dT/T)^2 |f| times the exponent's second derivative, is allowed as
  // 1e-12 |f| (it also covers the rounding of the two differences)
  const double g = de / f;
  const double e = std::fabs(ds - de) / ((std::fabs(g) + 1e-5) * std::fabs(de) + 1e-12 * std::fabs(f));
  return (e == e) ? e : 1e300;
}
void upd(double& e, double v) {
  if (!(v <= e)) e = v;
}
}  // namespace

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  FILE* fh = fopen(argv[1], "rb");
  if (!fh) return 3;
  int64_t n = 0;
  if (fread(&n, 8, 1, fh) != 1 || n <= 0) return 4;
  std::vector<double> in(12 * (size_t)n);
  if (fread(in.data(), 8, in.size(), fh) != in.size()) return 5;
  fclose(fh);
  auto col = [&](int k) { return in.data() + (size_t)k * n; };
  DevParams p{1.0, 2.73, 1.0, 1.0, 1.0 / 3.0, 0.1, 1e-3, 1e-12, 1e-6, 1.0, 50, 1000000, 0};
  // off the kinks of the clamped factors (10 K and 1e4 K), where the one-sided change and
  // the derivative legitimately differ
  const double temps[11] = {12.0, 30.0, 100.0, 300.0, 1e3, 3e3, 9e3, 3e4, 1e5, 1e6, 1e7};
  const unsigned flag_sets[2] = {0u, FL_CONST_KGR | FL_NO_ROVIB | FL_NO_CIE};
  double e_chem[NCHEM] = {0}, e_cool[NCOOL] = {0};
  double e_lpsi = 0, e_cxe = 0, e_cxcp = 0, e_clp = 0;
  long long checks = 0;
  for (int64_t i = 0; i < n; ++i) {
    const CellC<double> c = make_cell(col(0)[i], col(1)[i], col(2)[i], col(3)[i], col(4)[i], col(5)[i], col(6)[i],
                                      col(7)[i], col(8)[i], p);
    for (int t = 0; t < 12; ++t) {
      const double T = (t == 0) ? col(9)[i] : temps[t - 1];
      for (unsigned flags : flag_sets) {
        const double T1 = T * (1.0 + 1e-7);
        const ChemT<double> b = chem_T(c, T, flags);
        const CoolT<double> k = cool_T(c, b, flags);
        const ChemT<double> be = chem_T(c, T1, flags);
        const CoolT<double> ke = cool_T(c, be, flags);
        ChemT<double> bs;
        CoolT<double> ks;
        temp_blocks_step(c, b, k, T1, flags, bs, ks);
        const double* f0 = reinterpret_cast<const double*>(&b);
        const double* fe = reinterpret_cast<const double*>(&be);
        const double* fs = reinterpret_cast<const double*>(&bs);
        for (int j = 0; j < NCHEM; ++j) upd(e_chem[j], field_err(f0[j], fe[j], fs[j]));
        f0 = reinterpret_cast<const double*>(&k);
        fe = reinterpret_cast<const double*>(&ke);
        fs = reinterpret_cast<const double*>(&ks);
        for (int j = 0; j < NCOOL; ++j) upd(e_cool[j], field_err(f0[j], fe[j], fs[j]));
        // C/O/e root: converged from scratch, then capped at one step from 1e-7 off
        const double x2 = col(10)[i], xp = col(11)[i];
        const Equil<double> q = equilibrium(c, b, x2, xp, -1.0);
        const double lp = log_psi(c, b, q.xe);
        upd(e_lpsi, std::fabs(q.lpsi - lp) / std::fmax(std::fabs(lp), 1e-300));
        const Equil<double> qc = equilibrium(c, b, x2, xp, q.xe * (1.0 + 1e-7), 1);
        upd(e_cxe, std::fabs(qc.xe - q.xe) / q.xe);
        upd(e_cxcp, std::fabs(qc.xCp - q.xCp) / std::fmax(std::fabs(q.xCp), 1e-300));
        upd(e_clp, std::fabs(qc.lpsi - q.lpsi) / std::fmax(std::fabs(q.lpsi), 1e-300));
        ++checks;
      }
    }
  }
  printf("{\"checks\": %lld, \"lpsi_converged\": %.3e, \"capped_xe\": %.3e, \"capped_xCp\": %.3e, "
         "\"capped_lpsi\": %.3e", checks, e_lpsi, e_cxe, e_cxcp, e_clp);
  for (int j = 0; j < NCHEM; ++j) printf(", \"%s\": %.3e", kChemNames[j], e_chem[j]);
  for (int j = 0; j < NCOOL; ++j) printf(", \"%s\": %.3e", kCoolNames[j], e_cool[j]);
  printf("}\n");
  return 0;
}
