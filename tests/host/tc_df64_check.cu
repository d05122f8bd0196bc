// Host program that measures the error of the library's df64 (double-float) arithmetic
// and of its physics evaluated in df64, against FP64 (not part of libtc_gb300.so; built
// and run by tests/test_df64.py with the library's csrc/ on the include path).
//
// Usage: tc_df64_check IN
//   IN: n as int64, then 12 arrays of n doubles (n, chi_pe, chi_lw, f_shld_H2, f_shld_C,
//       F_LyC, xi, Z'_g, Z'_d, T, x_H2, x_H+), then dt as a double (unused).
// Prints one JSON object: the largest errors of each operation over seeded operands,
// and of each source term over the cells of IN.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "tc_phys.cuh"

using namespace tcg;

namespace {
uint64_t g_state = 0x9E3779B97F4A7C15ull;
double uniform() {  // splitmix64 -> [0, 1)
  uint64_t z = (g_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return double(z >> 11) * (1.0 / 9007199254740992.0);
}
double loguniform(double lo, double hi) { return std::exp(std::log(lo) + (std::log(hi) - std::log(lo)) * uniform()); }
double rel(double a, double b) { return std::fabs(a - b) / std::fmax(std::fabs(b), 1e-300); }
// running maximum that keeps a NaN (std::fmax would drop it)
void upd(double& e, double v) {
  if (!(v <= e)) e = v;
}
double out(double e) { return (e == e) ? e : 1e300; }  // NaN reported as 1e300
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

  // ---- arithmetic on seeded operands within FP32's range (relative to the FP64 result;
  // additions relative to the larger operand, since cancellation leaves only that
  // absolute accuracy); exp over [-70, 80], where its result is not subnormal in FP32
  // (closer to the underflow the trailing part loses bits), log in absolute terms
  double e_add = 0, e_mul = 0, e_div = 0, e_sqrt = 0, e_exp = 0, e_log = 0, e_conv = 0;
  for (int i = 0; i < 200000; ++i) {
    const double a = (uniform() < 0.5 ? -1 : 1) * loguniform(1e-15, 1e15);
    const double b = (uniform() < 0.5 ? -1 : 1) * loguniform(1e-15, 1e15);
    const double c = (uniform() < 0.5 ? -1 : 1) * std::fabs(a) * (1.0 + 1e-6 * (uniform() - 0.5));  // near-cancelling
    const df64 A(a), B(b), Cc(c);
    upd(e_conv, rel(double(A), a));
    upd(e_add, std::fabs(double(A + B) - (a + b)) / std::fmax(std::fabs(a), std::fabs(b)));
    upd(e_add, std::fabs(double(A + Cc) - (a + c)) / std::fmax(std::fabs(a), std::fabs(c)));
    upd(e_mul, rel(double(A * B), a * b));
    upd(e_div, rel(double(A / B), a / b));
    upd(e_sqrt, rel(double(m_sqrt(df64(std::fabs(a)))), std::sqrt(std::fabs(a))));
    const double x = -70.0 + 150.0 * uniform();
    const double xc = (i & 1) ? x : x * 1e-3;  // also small arguments
    upd(e_exp, rel(double(m_exp(df64(xc))), std::exp(xc)));
    const double y = loguniform(1e-30, 1e30);
    upd(e_log, std::fabs(double(m_log(df64(y))) - std::log(y)));
  }
  // saturation instead of infinities
  const bool sat_ok = double(df64(INFINITY)) == double(float(DF_BIG)) &&
                      std::fabs(double(m_exp(df64(1000.0))) / std::exp(80.0) - 1.0) < 1e-12;
  const bool under_ok = double(m_exp(df64(-100.0))) == 0.0 && double(m_log(df64(0.0))) == -double(float(DF_BIG));

  // ---- the physics in df64 against FP64 at the states of IN
  DevParams p{1.0, 2.73, 1.0, 1.0, 1.0 / 3.0, 0.1, 1e-3, 1e-12, 1e-6, 1.0, 50, 1000000, 0};
  double e_G = 0, e_L = 0, e_H = 0, e_form = 0, e_dest = 0, e_ion = 0, e_rec = 0, e_xe = 0, e_Td = 0;
  double e_chem = 0, e_cool = 0;
  for (int64_t i = 0; i < n; ++i) {
    const CellC<double> c = make_cell(col(0)[i], col(1)[i], col(2)[i], col(3)[i], col(4)[i], col(5)[i], col(6)[i],
                                      col(7)[i], col(8)[i], p);
    const CellC<df64> cd = cast_cell<df64>(c);
    const double T = col(9)[i], x2 = col(10)[i], xp = col(11)[i], xH = 1.0 - 2.0 * x2 - xp;
    const ChemT<double> b = chem_T(c, T, 0u);
    const ChemT<df64> bd = chem_T(cd, df64(T), 0u);
    upd(e_chem, rel(double(bd.kci), b.kci) * (b.kci > 1e-30));
    upd(e_chem, rel(double(bd.arr), b.arr));
    upd(e_chem, rel(double(bd.S), b.S) * (b.S > 1e-30));
    const CoolT<double> k = cool_T(c, b, 0u);
    const CoolT<df64> kd = cool_T(cd, bd, 0u);
    upd(e_cool, rel(double(kd.lyaE), k.lyaE) * (k.lyaE > 1e-30));
    upd(e_cool, rel(double(kd.nebT), k.nebT) * (k.nebT > 1e-30));
    upd(e_cool, rel(double(kd.rvLLTE), k.rvLLTE) * (k.rvLLTE > 1e-30));
    const Equil<double> q = equilibrium(c, b, x2, xp, -1.0);
    const Equil<df64> qd = equilibrium(cd, bd, df64(x2), df64(xp), df64(-1.0));
    upd(e_xe, rel(double(qd.xe), q.xe));
    const Src<double> s = source(c, b, k, x2, xp, xH, q, -1.0, -1.0);
    const Src<df64> sd = source(cd, bd, kd, df64(x2), df64(xp), df64(xH), qd, df64(-1.0), df64(-1.0));
    const double nn = c.n;
    upd(e_G, rel(double(sd.G), s.G));
    upd(e_L, rel(double(sd.L), s.L));
    upd(e_H, std::fabs(double(sd.H) - s.H) / (nn * std::fabs(s.G) + nn * nn * std::fabs(s.L)));
    upd(e_form, rel(double(sd.form), s.form) * (s.form > 1e-300));
    upd(e_dest, rel(double(sd.dest), s.dest) * (s.dest > 1e-300));
    upd(e_ion, rel(double(sd.ion), s.ion) * (s.ion > 1e-300));
    upd(e_rec, rel(double(sd.rec), s.rec) * (s.rec > 1e-300));
    upd(e_Td, rel(double(sd.Td), s.Td));
  }
  printf("{\"add\": %.3e, \"mul\": %.3e, \"div\": %.3e, \"sqrt\": %.3e, \"exp\": %.3e, \"log_abs\": %.3e, "
         "\"conv\": %.3e, \"saturates\": %s, \"underflow\": %s, \"chem_T\": %.3e, \"cool_T\": %.3e, \"xe\": %.3e, "
         "\"G\": %.3e, \"L\": %.3e, \"H\": %.3e, \"form\": %.3e, \"dest\": %.3e, \"ion\": %.3e, \"rec\": %.3e, "
         "\"Td\": %.3e, \"cells\": %lld}\n",
         out(e_add), out(e_mul), out(e_div), out(e_sqrt), out(e_exp), out(e_log), out(e_conv),
         sat_ok ? "true" : "false", under_ok ? "true" : "false", out(e_chem), out(e_cool), out(e_xe), out(e_G),
         out(e_L), out(e_H), out(e_form), out(e_dest), out(e_ion), out(e_rec), out(e_Td), (long long)n);
  return 0;
}
