// Host program that counts the FP64 arithmetic of the step as the library performs it
// (not part of libtc_gb300.so; built and run by paper_2210_08024_gb300/work.py).
//
// Two passes (FP64, FP32 and df64 calls counted separately):
//  1. cost per call: each building block of the step (the two temperature blocks, one
//     C/O/e root iteration and its set-up, one dust-temperature iteration and its
//     set-up, the source terms) is instantiated with a counting scalar and evaluated
//     once; the counts by operation class are its cost per call;
//  2. calls per cell: the library's own step functions, compiled here for the host,
//     advance a sample of cells in each mode while hooks count the calls and inner
//     iterations of every block (FP64 and FP32 separately).
// FP64 work per cell = sum over blocks of calls x cost, plus the hand-counted dense
// linear algebra of each Newton iteration (stated below).  Output: JSON on stdout.
//
// Input file: 12 arrays of n doubles (n, chi_pe, chi_lw, f_h2, f_c, F_lyc, xi, Zg, Zd,
// T, xH2, xHp), preceded by n as int64, then dt as a double.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace wc {
struct Calls {
  long long chem_T, cool_T, temp_step, equil, equil_it, dust, dust_it, source;
  long long newton64_it, chord64_it, newton32_it, polish_it, substep_paper, picard_it;
};
Calls calls[3];  // [0] FP64, [1] FP32, [2] df64 (double-float)
}  // namespace wc

#ifdef __CUDA_ARCH__
#define TCG_COUNT(name)
#define TCG_COUNT_D(name)
#else
#define TCG_COUNT(name) (::wc::calls[::tcg::Prec<F>::cls].name++)
#define TCG_COUNT_D(name) (::wc::calls[0].name++)
#endif

#include "tc_kernels.cuh"

// ------------------------------------------------------------------ counting scalar
namespace tcg {
struct OpCnt {
  long long add, mul, div, sqrt, exp, log;
};
static OpCnt g_ops;

struct CntD {
  double v;
  CntD() = default;
  constexpr CntD(double x) : v(x) {}
};
static_assert(sizeof(CntD) == 8, "counting scalar must look like a double");
template <> struct Prec<CntD> {
  static constexpr double root_tol = 1e-14;
  static constexpr bool fp32_range = false;
  static constexpr int cls = 0;
};
inline CntD operator+(CntD a, CntD b) { ++g_ops.add; return CntD(a.v + b.v); }
inline CntD operator-(CntD a, CntD b) { ++g_ops.add; return CntD(a.v - b.v); }
inline CntD operator*(CntD a, CntD b) { ++g_ops.mul; return CntD(a.v * b.v); }
inline CntD operator/(CntD a, CntD b) { ++g_ops.div; return CntD(a.v / b.v); }
inline CntD operator-(CntD a) { return CntD(-a.v); }
inline CntD& operator+=(CntD& a, CntD b) { a = a + b; return a; }
inline bool operator<(CntD a, CntD b) { return a.v < b.v; }
inline bool operator>(CntD a, CntD b) { return a.v > b.v; }
inline bool operator<=(CntD a, CntD b) { return a.v <= b.v; }
inline bool operator>=(CntD a, CntD b) { return a.v >= b.v; }
inline bool operator==(CntD a, CntD b) { return a.v == b.v; }
inline CntD m_exp(CntD x) { ++g_ops.exp; return CntD(std::exp(x.v)); }
inline CntD m_log(CntD x) { ++g_ops.log; return CntD(std::log(x.v)); }
inline CntD m_sqrt(CntD x) { ++g_ops.sqrt; return CntD(std::sqrt(x.v)); }
inline CntD m_max(CntD a, CntD b) { ++g_ops.add; return CntD(std::fmax(a.v, b.v)); }
inline CntD m_min(CntD a, CntD b) { ++g_ops.add; return CntD(std::fmin(a.v, b.v)); }
inline CntD m_abs(CntD a) { return CntD(std::fabs(a.v)); }
}  // namespace tcg

using namespace tcg;

static OpCnt diff(const OpCnt& a, const OpCnt& b) {
  return OpCnt{a.add - b.add, a.mul - b.mul, a.div - b.div, a.sqrt - b.sqrt, a.exp - b.exp, a.log - b.log};
}
static void print_ops(const char* name, const OpCnt& o, double scale, bool comma) {
  printf("  \"%s\": {\"add\": %.3f, \"mul\": %.3f, \"div\": %.3f, \"sqrt\": %.3f, \"exp\": %.3f, \"log\": %.3f}%s\n",
         name, o.add * scale, o.mul * scale, o.div * scale, o.sqrt * scale, o.exp * scale, o.log * scale,
         comma ? "," : "");
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* fh = fopen(argv[1], "rb");
  if (!fh) return 3;
  int64_t n = 0;
  double dt = 0;
  if (fread(&n, 8, 1, fh) != 1 || n <= 0) return 4;
  std::vector<double> a(12 * n);
  if (fread(a.data(), 8, a.size(), fh) != a.size() || fread(&dt, 8, 1, fh) != 1) return 5;
  fclose(fh);
  auto col = [&](int k) { return a.data() + (size_t)k * n; };
  DevParams p{1.0, 2.73, 1.0, 1.0, 1.0 / 3.0, 0.1, 1e-3, 1e-12, 1e-6, 1.0, 50, 1000000, 0};  // library defaults

  // ---- pass 1: cost per call of each block (FP64), averaged over the sample's cells
  OpCnt c_chem{}, c_cool{}, c_step{}, c_src{}, c_eq_set{}, c_eq_it{}, c_dust_set{}, c_dust_it{};
  long long nb = 0;
  for (int64_t i = 0; i < n; i += (n > 256 ? n / 256 : 1), ++nb) {
    CellC<double> cd = make_cell(col(0)[i], col(1)[i], col(2)[i], col(3)[i], col(4)[i], col(5)[i], col(6)[i],
                                 col(7)[i], col(8)[i], p);
    CellC<CntD> c = cast_cell<CntD>(cd);
    const double T = col(9)[i], x2 = col(10)[i], xp = col(11)[i];
    OpCnt o0 = g_ops;
    ChemT<CntD> b = chem_T(c, CntD(T), 0u);
    OpCnt o1 = g_ops;
    CoolT<CntD> k = cool_T(c, b, 0u);
    OpCnt o2 = g_ops;
    {  // the temperature blocks stepped to T + 1e-7 T (the Jacobian's temperature column)
      ChemT<CntD> bT;
      CoolT<CntD> kT;
      const OpCnt s0 = g_ops;
      temp_blocks_step(c, b, k, CntD(T * (1.0 + 1e-7)), 0u, bT, kT);
      const OpCnt d = diff(g_ops, s0);
      c_step.add += d.add; c_step.mul += d.mul; c_step.div += d.div;
      c_step.sqrt += d.sqrt; c_step.exp += d.exp; c_step.log += d.log;
      g_ops = s0;  // keep the differences below to the blocks they time
      o2 = g_ops;
    }
    // C/O/e root: a cold solve (k iterations) and a warm one from the root (1 iteration)
    long long it0 = wc::calls[0].equil_it;
    Equil<CntD> q = equilibrium(c, b, CntD(x2), CntD(xp), CntD(-1.0));
    long long kc = wc::calls[0].equil_it - it0;
    OpCnt o3 = g_ops;
    it0 = wc::calls[0].equil_it;
    equilibrium(c, b, CntD(x2), CntD(xp), q.xe);
    long long kw = wc::calls[0].equil_it - it0;
    OpCnt o4 = g_ops;
    // dust temperature: cold and warm
    long long d0 = wc::calls[0].dust_it;
    CntD Td = dust_T(c, b.T, b.sqT, CntD(-1.0));
    long long dc = wc::calls[0].dust_it - d0;
    OpCnt o5 = g_ops;
    d0 = wc::calls[0].dust_it;
    dust_T(c, b.T, b.sqT, Td);
    long long dw = wc::calls[0].dust_it - d0;
    OpCnt o6 = g_ops;
    // source terms with the dust temperature frozen (its root counted separately)
    source(c, b, k, CntD(x2), CntD(xp), CntD(1.0 - 2.0 * x2 - xp), q, Td, CntD(-1.0));
    OpCnt o7 = g_ops;
    auto acc = [](OpCnt& s, const OpCnt& d) {
      s.add += d.add; s.mul += d.mul; s.div += d.div; s.sqrt += d.sqrt; s.exp += d.exp; s.log += d.log;
    };
    acc(c_chem, diff(o1, o0));
    acc(c_cool, diff(o2, o1));
    acc(c_src, diff(o7, o6));
    OpCnt ecold = diff(o3, o2), ewarm = diff(o4, o3), dcold = diff(o5, o4), dwarm = diff(o6, o5);
    if (kc > kw) {  // per-iteration cost from the difference, set-up from the warm solve
      OpCnt per{(ecold.add - ewarm.add) / (kc - kw), (ecold.mul - ewarm.mul) / (kc - kw),
                (ecold.div - ewarm.div) / (kc - kw), (ecold.sqrt - ewarm.sqrt) / (kc - kw),
                (ecold.exp - ewarm.exp) / (kc - kw), (ecold.log - ewarm.log) / (kc - kw)};
      acc(c_eq_it, per);
      acc(c_eq_set, OpCnt{ewarm.add - kw * per.add, ewarm.mul - kw * per.mul, ewarm.div - kw * per.div,
                          ewarm.sqrt - kw * per.sqrt, ewarm.exp - kw * per.exp, ewarm.log - kw * per.log});
    } else {
      acc(c_eq_set, ewarm);
    }
    if (dc > dw) {
      OpCnt per{(dcold.add - dwarm.add) / (dc - dw), (dcold.mul - dwarm.mul) / (dc - dw),
                (dcold.div - dwarm.div) / (dc - dw), 0, 0, 0};
      acc(c_dust_it, per);
      acc(c_dust_set, OpCnt{dwarm.add - dw * per.add, dwarm.mul - dw * per.mul, dwarm.div - dw * per.div,
                            dwarm.sqrt, dwarm.exp, dwarm.log});
    } else {
      acc(c_dust_set, dwarm);
    }
  }
  const double inv = 1.0 / (double)nb;

  // ---- pass 2: calls per cell in each mode
  printf("{\n  \"cells\": %lld,\n  \"dt_s\": %.6e,\n", (long long)n, dt);
  print_ops("cost_chem_T", c_chem, inv, true);
  print_ops("cost_cool_T", c_cool, inv, true);
  print_ops("cost_temp_step", c_step, inv, true);
  print_ops("cost_source", c_src, inv, true);
  print_ops("cost_equil_setup", c_eq_set, inv, true);
  print_ops("cost_equil_iter", c_eq_it, inv, true);
  print_ops("cost_dust_setup", c_dust_set, inv, true);
  print_ops("cost_dust_iter", c_dust_it, inv, true);
  for (int mode = 0; mode <= 2; ++mode) {
    wc::calls[0] = wc::Calls{};
    wc::calls[1] = wc::Calls{};
    wc::calls[2] = wc::Calls{};
    long long nsub = 0;
    for (int64_t i = 0; i < n; ++i) {
      CellC<double> c = make_cell(col(0)[i], col(1)[i], col(2)[i], col(3)[i], col(4)[i], col(5)[i], col(6)[i],
                                  col(7)[i], col(8)[i], p);
      CellC<float> cf = cast_cell<float>(c);
      CellC<df64> cd = cast_cell<df64>(c);
      LaneState s;
      s.t = 0; s.xH2 = col(10)[i]; s.xHp = col(11)[i]; s.Td = -1; s.nsub = 0; s.status = 0; s.iters = 0;
      if (mode == 2) {  // the mixed kernels solve the initial equilibrium in df64
        ChemT<df64> b0 = chem_T(cd, df64(col(9)[i]), p.flags);
        Equil<df64> q0 = equilibrium(cd, b0, df64(s.xH2), df64(s.xHp), df64(-1.0));
        s.xe = double(q0.xe); s.xCp = double(q0.xCp); s.xCO = double(q0.xCO);
      } else {
        ChemT<double> b0 = chem_T(c, col(9)[i], p.flags);
        Equil<double> q0 = equilibrium(c, b0, s.xH2, s.xHp, -1.0);
        s.xe = q0.xe; s.xCp = q0.xCp; s.xCO = q0.xCO;
      }
      s.mu = c.muH / (1.1 + s.xe - s.xH2);
      s.Tmu = col(9)[i] / s.mu;
      double xg = s.xe, tg = -1.0;
      df64 thp = df64(-1.0);
      float xgf = (float)s.xe, tgf = -1.f;
      while (s.t < dt && s.nsub < p.max_sub) {
        if (mode == 0) substep_paper(c, p, dt, s);
        else if (mode == 1) substep_newton64(c, p, dt, s, xg, tg);
        else substep_mixed(c, cd, cf, p, dt, s, xgf, tgf, thp);
        if (!finite3(s.Tmu, s.xH2, s.xHp)) break;
      }
      nsub += s.nsub;
    }
    const wc::Calls& k = wc::calls[0];
    const wc::Calls& f = wc::calls[1];
    const wc::Calls& h = wc::calls[2];
    printf("  \"mode%d\": {\"substeps\": %.4f, \"fp64\": {\"chem_T\": %.4f, \"cool_T\": %.4f, \"temp_step\": %.4f, \"equil\": %.4f, "
           "\"equil_it\": %.4f, \"dust\": %.4f, \"dust_it\": %.4f, \"source\": %.4f, \"newton64_it\": %.4f, "
           "\"chord64_it\": %.4f, \"newton32_it\": %.4f, \"polish_it\": %.4f, \"substep_paper\": %.4f, "
           "\"picard_it\": %.4f}, ",
           mode, (double)nsub / n, (double)k.chem_T / n, (double)k.cool_T / n, (double)k.temp_step / n, (double)k.equil / n,
           (double)k.equil_it / n, (double)k.dust / n, (double)k.dust_it / n, (double)k.source / n,
           (double)k.newton64_it / n, (double)k.chord64_it / n, (double)k.newton32_it / n, (double)k.polish_it / n,
           (double)k.substep_paper / n, (double)k.picard_it / n);
    for (int cl = 1; cl <= 2; ++cl) {
      const wc::Calls& x = (cl == 1) ? f : h;
      printf("\"%s\": {\"chem_T\": %.4f, \"cool_T\": %.4f, \"temp_step\": %.4f, \"equil\": %.4f, \"equil_it\": %.4f, \"dust\": %.4f, "
             "\"dust_it\": %.4f, \"source\": %.4f}%s",
             (cl == 1) ? "fp32" : "df64", (double)x.chem_T / n, (double)x.cool_T / n, (double)x.temp_step / n,
             (double)x.equil / n,
             (double)x.equil_it / n, (double)x.dust / n, (double)x.dust_it / n, (double)x.source / n,
             (cl == 1) ? ", " : "");
    }
    printf("}%s\n", mode < 2 ? "," : "");
  }
  printf("}\n");
  return 0;
}
