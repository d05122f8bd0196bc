// Device physics of the thermochemistry source step (arXiv:2210.08024, Secs. 3-4).
//
// Organised for the GPU rather than term by term:
//   CellC<F>   per-cell constants: density and radiation are frozen over the step
//              (Sec. 6.1), so every quantity that depends only on them is built once.
//   ChemT<F>   temperature-only pieces of the chemistry and of the C/O/e equilibrium,
//              evaluated once per temperature and shared by both.
//   CoolT<F>   temperature-only pieces of the heating and cooling functions.
// Powers of T and psi are taken as exp(c ln T), exp(c ln psi) from one logarithm.
//
// F is double for the FP64 paths, float for the mixed path's Newton iterations and df64
// (double-float, tc_df64.cuh) for its high-precision evaluations.  Terms
// the paper names but does not print (closures: cited fits and tables it does not
// reproduce) use one stated definition each, labelled where it is a stand-in for the
// cited source; the CPU checker uses the same definitions, written independently.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tc_df64.cuh"

// Physics and substep functions are host+device so the host compiler can also build
// them (used by the host-side test harness of the library's own kernels).
#ifndef TCG_FN
#define TCG_FN __host__ __device__ __forceinline__
#endif
// The four large blocks (temperature factors, cooling factors, the C/O/e equilibrium
// and the source terms) stay out of line: the step kernel calls each from several
// places, and inlining them all makes the kernel larger than the instruction cache
// (instruction-fetch stalls dominated) and raises register use.  Out of line the FP64
// Newton step runs 1.44x faster.
#ifndef TCG_BIG
#define TCG_BIG __host__ __device__ __noinline__
#endif
// Work-counting hooks: empty in the library; the host work counter (tc_workcount.cu)
// defines them to count calls and inner iterations of the step's building blocks.
// TCG_COUNT is used inside templates on the scalar type F; TCG_COUNT_D in FP64 code.
#ifndef TCG_COUNT
#define TCG_COUNT(name)
#endif
#ifndef TCG_COUNT_D
#define TCG_COUNT_D(name)
#endif

namespace tcg {

// ------------------------------------------------------------------ constants (cgs)
constexpr double KB = 1.380649e-16;
constexpr double EV = 1.602176634e-12;
constexpr double CLIGHT = 2.99792458e10;
constexpr double ARAD = 7.57e-15;  // as printed in Sec. 4.3.6
constexpr double PC_CM = 3.0856775814913673e18;
constexpr double LN10 = 2.302585092994046;
constexpr double FOURPI = 12.566370614359172;

constexpr unsigned FL_CONST_KGR = 1u, FL_NO_ROVIB = 2u, FL_NO_CIE = 4u;

// ------------------------------------------------------------------ precision-generic math
// FP64 exp and log are called out of line on the device: the physics blocks hold ~50
// call sites, and one shared copy keeps the kernels' code smaller (instruction fetch;
// FP64 Newton step on the 128^3 slab 232.5 -> 226.5 ms).
__device__ __noinline__ inline double m_exp64_ool(double x) { return exp(x); }
__device__ __noinline__ inline double m_log64_ool(double x) { return log(x); }
TCG_FN double m_exp(double x) {
#ifdef __CUDA_ARCH__
  return m_exp64_ool(x);
#else
  return exp(x);
#endif
}
TCG_FN float m_exp(float x) { return expf(x); }
TCG_FN double m_log(double x) {
#ifdef __CUDA_ARCH__
  return m_log64_ool(x);
#else
  return log(x);
#endif
}
TCG_FN float m_log(float x) { return logf(x); }
TCG_FN double m_sqrt(double x) { return sqrt(x); }
TCG_FN float m_sqrt(float x) { return sqrtf(x); }
TCG_FN double m_max(double a, double b) { return fmax(a, b); }
TCG_FN float m_max(float a, float b) { return fmaxf(a, b); }
TCG_FN double m_min(double a, double b) { return fmin(a, b); }
TCG_FN float m_min(float a, float b) { return fminf(a, b); }
TCG_FN double m_abs(double a) { return fabs(a); }
TCG_FN float m_abs(float a) { return fabsf(a); }

// Precision traits of the scalar types: the relative tolerance of the inner root solves
// (C/O/e equilibrium, dust temperature), a little above each type's rounding; whether
// the type has only FP32's exponent range; and its class for the work counter
// (0 FP64, 1 FP32, 2 df64).
template <class F> struct Prec;
template <> struct Prec<double> {
  static constexpr double root_tol = 1e-14;
  static constexpr bool fp32_range = false;
  static constexpr int cls = 0;
};
template <> struct Prec<float> {
  static constexpr double root_tol = 1e-7;
  static constexpr bool fp32_range = true;
  static constexpr int cls = 1;
};
template <> struct Prec<df64> {
  static constexpr double root_tol = 1e-12;
  static constexpr bool fp32_range = true;
  static constexpr int cls = 2;
};

// A value computed at run time, in precision F (df64 keeps subnormal trailing parts on
// the device; constants convert at compile time with F(x)).
template <class F> TCG_FN F to_prec(double x) { return F(x); }
template <> TCG_FN df64 to_prec<df64>(double x) { return to_df64(x); }

template <class F> TCG_FN F logistic(F z) { return F(1) / (F(1) + m_exp(-z)); }

// Parameters copied to the device by value with each launch.
struct MlpMma;  // seed network in the tensor-core layout (tc_mlp_mma.cuh)

struct DevParams {
  double dvdr_kms_pc, T_cmb, chi0, opt_over_fuv, tau_ratio;
  double limiter, fd_rel, rtol, rtol_mixed, T_floor;
  int newton_max, max_sub;
  unsigned flags;
  const unsigned* order = nullptr;  // optional: the k-th claimed cell is order[k] (cost-ordered queue)
  const MlpMma* mlp_mma = nullptr;  // seeded modes: the network for the warp-level inference
};

// ------------------------------------------------------------------ per-cell constants
template <class F> struct CellC {
  F n, lnn;
  F G0;                 // 1.7 chi_FUV (Sec. 4.2, Eq. e:chi_FUV)
  F zpd;                // 5.7e-11 chi_LW f_shld,H2 (Eq. eq:H2_pd)
  F zpiH, zpiH2;        // 3.1e-18 F, 4.6e-18 F (Eqs. e:H_pi, eq:H2_pi)
  F zpiC_rad, zcrC;     // 3.43e-10 chi_LW f_shld,C ; 3.85 xi (Sec. 3.2.1)
  F xi;
  F rCO2;               // (n_CO,crit / n)^2 (Eqs. e:CO, e:CO_fit), +inf without CRs or dust
  F qH2;                // q_cr,H2(n) in erg
  F xCtot, xOtot, Zg, Zd;
  F NtX;                // n_H / |dv/dr| [cm^-2 (km/s)^-1]
  F Gd;                 // dust radiative heating per H
  F Bd;                 // sigma_IR c a / T_d^2 = 2e-27 Z'_d c a
  F Cgd;                // n 3.2e-34 Z'_d (times sqrt(T) gives the gas-dust coupling)
  F Tc, Tc4, Td_hi;     // T_cmb, T_cmb^4, (2 Gd / B)^(1/6)
  F xMH_pref;           // sqrt(1.67 xi / n) (molecular-ion electrons)
  F K, muH;             // K = n mu_H k_B/(gamma-1) (Eq. e:ODE1), mu_H (Table 1)
};

// Builds the per-cell constants in FP64 (always), then converts.
TCG_FN CellC<double> make_cell(double n, double chi_pe, double chi_lw, double fh2, double fc,
                                                   double Flyc, double xi, double Zg, double Zd,
                                                   const DevParams& p, double chi0_cell = -1.0) {
  // chi0: the unattenuated FUV scale of the optical dust heating; per cell when given
  // (driver runs with several radiation scales in one launch), else the launch's.
  const double chi0 = (chi0_cell >= 0.0) ? chi0_cell : p.chi0;
  CellC<double> c;
  c.n = n;
  c.lnn = log(n);
  c.G0 = 1.7 * (1.8e-4 * chi_pe + 3.0e-5 * chi_lw) / 2.1e-4;
  c.zpd = 5.7e-11 * chi_lw * fh2;
  c.zpiH = 3.1e-18 * Flyc;
  c.zpiH2 = 4.6e-18 * Flyc;
  c.zpiC_rad = 3.43e-10 * chi_lw * fc;
  c.zcrC = 3.85 * xi;
  c.xi = xi;
  if (xi > 0.0 && Zd > 0.0) {
    double xi16 = xi * 1e16;
    double lnZd = log(Zd);
    double chi13 = (chi_lw > 0.0) ? exp(log(chi_lw) / 3.0) : 0.0;
    double lnCOc = chi13 * (log(4e3) + lnZd - 2.0 * log(xi16)) + (log(50.0 * xi16) - 1.4 * lnZd);
    c.rCO2 = exp(2.0 * (lnCOc - c.lnn));
  } else {
    c.rCO2 = INFINITY;
  }
  double l10n = c.lnn / LN10;  // q_cr,H2: 10 -> 13 -> 17 -> 18 eV, linear in log10 n
  double q = (l10n < 2.0) ? 10.0
           : (l10n < 4.0) ? 10.0 + 1.5 * (l10n - 2.0)
           : (l10n < 7.0) ? 13.0 + (4.0 / 3.0) * (l10n - 4.0)
           : (l10n < 10.0) ? 17.0 + (l10n - 7.0) / 3.0 : 18.0;
  c.qH2 = q * EV;
  c.xCtot = 1.6e-4 * Zg;
  c.xOtot = 3.2e-4 * Zg;
  c.Zg = Zg;
  c.Zd = Zd;
  c.NtX = (p.dvdr_kms_pc > 0.0) ? n * (PC_CM / p.dvdr_kms_pc) : INFINITY;
  // dust heating: absorption of PE, LW (c E = 4 pi J) and LyC photons (Sec. 4.3.6 with
  // the Sec. 2.4 cross sections) and the attenuated optical band.
  double g = Zd * (FOURPI * (0.9e-21 * 1.8e-4 * chi_pe + 1.5e-21 * 3.0e-5 * chi_lw) + 1.9e-21 * 19.4 * EV * Flyc);
  if (p.opt_over_fuv > 0.0 && chi0 > 0.0) {
    double ratio = fmin(chi_pe / chi0, 1.0);
    double att = (ratio > 0.0) ? exp(p.tau_ratio * log(ratio)) : 0.0;
    g += 0.3e-21 * Zd * p.opt_over_fuv * FOURPI * 2.1e-4 * chi0 * att;
  }
  c.Gd = g;
  c.Bd = 2e-27 * Zd * CLIGHT * ARAD;
  c.Cgd = n * 3.2e-34 * Zd;
  c.Tc = p.T_cmb;
  c.Tc4 = p.T_cmb * p.T_cmb * p.T_cmb * p.T_cmb;
  c.Td_hi = (Zd > 0.0 && g > 0.0) ? exp(log(2.0 * g / c.Bd) / 6.0) : 0.0;
  c.xMH_pref = (xi > 0.0) ? sqrt(1.67 * xi / n) : 0.0;
  c.muH = 1.40 - 0.02 * (Zg - 1.0);
  c.K = n * c.muH * KB / (2.0 / 3.0);
  return c;
}

template <class F> TCG_FN CellC<F> cast_cell(const CellC<double>& d) {
  CellC<F> c;
  c.n = to_prec<F>(d.n); c.lnn = to_prec<F>(d.lnn); c.G0 = to_prec<F>(d.G0); c.zpd = to_prec<F>(d.zpd); c.zpiH = to_prec<F>(d.zpiH); c.zpiH2 = to_prec<F>(d.zpiH2);
  c.zpiC_rad = to_prec<F>(d.zpiC_rad); c.zcrC = to_prec<F>(d.zcrC); c.xi = to_prec<F>(d.xi); c.rCO2 = to_prec<F>(d.rCO2); c.qH2 = to_prec<F>(d.qH2);
  c.xCtot = to_prec<F>(d.xCtot); c.xOtot = to_prec<F>(d.xOtot); c.Zg = to_prec<F>(d.Zg); c.Zd = to_prec<F>(d.Zd); c.NtX = to_prec<F>(d.NtX); c.Gd = to_prec<F>(d.Gd);
  c.Bd = to_prec<F>(d.Bd); c.Cgd = to_prec<F>(d.Cgd); c.Tc = to_prec<F>(d.Tc); c.Tc4 = to_prec<F>(d.Tc4); c.Td_hi = to_prec<F>(d.Td_hi);
  c.xMH_pref = to_prec<F>(d.xMH_pref); c.K = to_prec<F>(d.K); c.muH = to_prec<F>(d.muH);
  return c;
}

// ------------------------------------------------------------------ temperature blocks
// WD01c grain-recombination coefficient sets (C0..C6) for H+ and C+.
#define WDH0 12.25
#define WDH1 8.074e-6
#define WDH2 1.378
#define WDH3 5.087e2
#define WDH4 1.586e-2
#define WDH5 0.4723
#define WDH6 1.102e-5
#define WDC0 45.58
#define WDC1 6.089e-3
#define WDC2 1.128
#define WDC3 4.331e2
#define WDC4 4.845e-2
#define WDC5 0.8120
#define WDC6 1.333e-4

template <class F> struct ChemT {
  F T, lnT, sqT, invT;
  F S;                 // cooling/electron sigmoid of Sec. 4.3
  F kgr;               // Eq. e:H2form (or constant)
  F arr;               // case-B alpha_rr,H+
  F kci;               // collisional ionisation of H
  F kcdH, kcdH2;       // collisional dissociation of H2
  F arrC, kCpH2;       // C+ recombination, C+ + H2
  F xMH_T;             // T-part of x_MH+: 1/sqrt(alpha_MH)
  F xe_hot;            // x_e,He,CIE + Z'_g x_e,metal,CIE
  F wdH3T, wdHex, wdC3T, wdCex;  // C3 T^C4 and -C5 - C6 ln T for H and C
};

// Electrons of hot gas at log10 T = lt: x_e,He,CIE (two logistic steps, at 4.45 and
// 4.95, whose exponentials differ by the constant factor exp(0.5/0.06)) + Z'_g
// x_e,metal,CIE (one step at 5.5).
template <class F> TCG_FN F xe_hot_of(const CellC<F>& c, F lt) {
  F eHe = m_exp((F(4.45) - lt) * F(1.0 / 0.06));
  F xeHe = F(0.1) * (F(1) / (F(1) + eHe) + F(1) / (F(1) + eHe * F(4160.262005375057)));  // exp(25/3)
  F xeMet = F(0.012) * logistic((lt - F(5.5)) * F(4));
  return xeHe + c.Zg * xeMet;
}

template <class F> TCG_BIG ChemT<F> chem_T(const CellC<F>& c, F T, unsigned flags) {
  TCG_COUNT(chem_T);
  ChemT<F> b;
  b.T = T;
  b.lnT = m_log(T);
  b.sqT = m_sqrt(T);
  const F invT = F(1) / T;
  b.invT = invT;
  b.S = F(1) / (F(1) + m_exp(F(-10.0 / 1.5e4) * (T - F(2.75e4))));
  if (flags & FL_CONST_KGR) {
    b.kgr = F(3.0e-17) * c.Zd;
  } else {
    F s2 = b.sqT * F(0.1);  // sqrt(T/100)
    F T2 = T * F(0.01);
    b.kgr = F(3.0e-17) * c.Zd * F(2) * s2 / (F(1) + F(0.4) * s2 + F(0.2) * T2 + F(0.08) * T2 * T2);
  }
  F lT4 = b.lnT - F(9.210340371976184);  // ln(T/1e4)
  b.arr = F(2.54e-13) * m_exp((F(-0.8163) - F(0.0208) * lT4) * lT4);
  b.kci = F(5.85e-11) * b.sqT * m_exp(F(-157809.1) * invT) / (F(1) + b.sqT * F(0.003162277660168379));
  b.kcdH = F(6.67e-12) * b.sqT * m_exp(F(-1) - F(63593.0) * invT);
  b.kcdH2 = F(5.996e-30) * m_exp(F(4.1881) * b.lnT - F(54657.4) * invT - F(5.6881) * m_log(F(1) + F(6.761e-6) * T));
  F lT300 = b.lnT - F(5.703782474656201);  // ln(T/300)
  b.arrC = F(4.67e-12) * m_exp(F(-0.6) * lT300);
  b.kCpH2 = F(4.0e-16) * m_exp(F(-0.2) * lT300);
  b.xMH_T = m_exp(F(0.345) * lT300) * F(2041.2414523193154);  // 1/sqrt(2.4e-7 (T/300)^-0.69)
  b.xe_hot = xe_hot_of(c, b.lnT * F(0.43429448190325176));  // at log10 T
  b.wdH3T = F(WDH3) * m_exp(F(WDH4) * b.lnT);
  b.wdHex = F(-WDH5) - F(WDH6) * b.lnT;
  b.wdC3T = F(WDC3) * m_exp(F(WDC4) * b.lnT);
  b.wdCex = F(-WDC5) - F(WDC6) * b.lnT;
  return b;
}

template <class F> struct CoolT {
  F fcA, fcB;          // k_H2*-H, k_H2*-H2 (H2* de-excitation for n_crit)
  F eps_num;           // 5.22 + 2.25 T^0.147
  F lyaE;              // E_21 k_12 (Eq. e:k_lya)
  F ffrr;              // free-free + case-B recombination cooling per x_e x_H+
  F cpke, cpkH, cpb;   // C+ 158um: k_e, k_H, Boltzmann factor g1/g0 exp(-E/T)
  F ok10, ob1, ob2, ob21;  // O: k10 and g-weighted Boltzmann factors
  F ck10, cb1, cb2, cb21;  // C
  F rvLlow, rvLLTE;    // H2 ro-vib: low-density and LTE per-molecule rates
  F coA, coN;          // CO stand-in: 4e-27 (T/10)^1.5 and 3e3 (T/10)^0.5
  F grT, grB;          // grain recombination cooling: 4.65e-30 T^0.94 and 0.74 T^-0.068
  F nebT, nebX;        // nebular: T-factor and density exponent (Eq. e:Lambda_neb)
  F cie;               // S-weighted CIE term: Lambda_He + Z'_g Lambda_metal
};

// Sums of several temperature factors in the cooling blocks, shared by cool_T and by
// temp_blocks_step (which evaluates them afresh at the stepped temperature).
// Ly-alpha (Eq. e:k_lya): E_21 5.31e-8 T4^0.15 / (1 + (T4/5)^0.65) exp(-11.84/T4) with
// E_21/k_B = 1.184e5 K, from ln(T/1e4) and 1e4/T.
template <class F> TCG_FN F lya_of(F lT4, F invT4) {
  return F(1.184e5 * KB * 5.31e-8) * m_exp(F(0.15) * lT4 - F(11.84) * invT4) /
         (F(1) + m_exp(F(0.65) * (lT4 - F(1.6094379124341003))));
}
// free-free Gaunt factor at log10 T = lt
template <class F> TCG_FN F gff_of(F lt) {
  F dg = F(5.5) - lt;
  return F(1.1) + F(0.34) * m_exp(-dg * dg * F(1.0 / 3.0));
}
// H2 ro-vibrational LTE rate per molecule from ln(T/1000) and 1000/T (T clamped to
// [10, 1e4] K by the caller): rotational and vibrational parts
template <class F> TCG_FN F rovib_lte_of(F lT3, F iT3) {
  F q = F(0.13) * iT3;
  F Lrot = F(9.5e-22) * m_exp(F(3.76) * lT3 - q * q * q) / (F(1) + F(0.12) * m_exp(F(2.1) * lT3)) +
           F(3e-24) * m_exp(F(-0.51) * iT3);
  F Lvib = F(6.7e-19) * m_exp(F(-5.86) * iT3) + F(1.6e-18) * m_exp(F(-11.7) * iT3);
  return Lrot + Lvib;
}
// CIE cooling of He and metals (before the S weighting) at log10 T = lt
template <class F> TCG_FN F cie_of(const CellC<F>& c, F lt) {
  F z1 = (lt - F(5.0)) * F(1.0 / 0.15), z2 = (lt - F(5.35)) * F(1.0 / 0.28), z3 = (lt - F(6.3)) * F(1.0 / 0.35);
  return F(2.0e-23) * m_exp(F(-0.5) * z1 * z1) +
         c.Zg * (F(5.4e-22) * m_exp(F(-0.5) * z2 * z2) + F(5.0e-23) * m_exp(F(-0.5) * z3 * z3));
}

template <class F> TCG_BIG CoolT<F> cool_T(const CellC<F>& c, const ChemT<F>& b, unsigned flags) {
  TCG_COUNT(cool_T);
  CoolT<F> k;
  const F T = b.T, lnT = b.lnT;
  const F invT = b.invT;
  k.fcA = F(1.0e-12) * b.sqT * m_exp(F(-1000.0) * invT);
  k.fcB = F(1.4e-12) * b.sqT * m_exp(F(-18100.0) / (T + F(1200.0)));
  k.eps_num = F(5.22) + F(2.25) * m_exp(F(0.147) * lnT);
  F lT4 = lnT - F(9.210340371976184);
  F invT4 = F(1e4) * invT;
  k.lyaE = lya_of(lT4, invT4);
  F lt = lnT * F(0.43429448190325176);
  k.ffrr = F(1.42e-27) * b.sqT * gff_of(lt) + b.arr * F(KB) * T * (F(0.684) - F(0.0416) * lT4);
  // C+ 158 um: n_e,crit = 53 T4^1/2, n_H,crit = 3e3 T2^(-0.1281 - 0.0087 ln T2), A = 2.3e-6
  F lT2 = lnT - F(4.605170185988092);
  k.cpke = F(2.3e-6 / 53.0 * 100.0) * b.sqT * invT;  // / (53 T^1/2 / 100)
  k.cpkH = F(2.3e-6 / 3e3) * m_exp((F(0.1281) + F(0.0087) * lT2) * lT2);
  k.cpb = F(2) * m_exp(F(-91.25) * invT);
  // O 3-level: n_crit(T) through 2.5e5 (10 K) and 4.9e4 (5000 K); C: 620 and 150
  F lT10 = lnT - F(2.302585092994046);
  const F sO = F(-0.2622274154608984);  // ln(4.9e4/2.5e5)/ln 500
  const F sC = F(-0.22834652828762741);  // ln(150/620)/ln 500
  k.ok10 = F(8.91e-5 / 2.5e5) * m_exp(-sO * lT10);
  // exp(-E2/T) = exp(-E1/T) exp(-(E2 - E1)/T): two exponentials for the three factors
  F eO1 = m_exp(F(-227.7) * invT), eO21 = m_exp(F(-(326.6 - 227.7)) * invT);
  k.ob1 = F(3.0 / 5.0) * eO1;
  k.ob2 = F(1.0 / 5.0) * (eO1 * eO21);
  k.ob21 = F(1.0 / 3.0) * eO21;
  k.ck10 = F(7.93e-8 / 620.0) * m_exp(-sC * lT10);
  F eC1 = m_exp(F(-23.6) * invT), eC21 = m_exp(F(-(62.4 - 23.6)) * invT);
  k.cb1 = F(3.0) * eC1;
  k.cb2 = F(5.0) * (eC1 * eC21);
  k.cb21 = F(5.0 / 3.0) * eC21;
  // H2 ro-vibrational: T clamped to [10, 1e4] K (equivalently ln T clamped)
  if (flags & FL_NO_ROVIB) {
    k.rvLlow = F(0); k.rvLLTE = F(1);
  } else {
    F lnTc = m_min(m_max(lnT, F(2.302585092994046)), F(9.210340371976184));
    F x = lnTc * F(0.43429448190325176);
    F poly = F(-103.0) + x * (F(97.59) + x * (F(-48.05) + x * (F(10.80) + x * F(-0.9032))));
    k.rvLlow = m_exp(poly * F(LN10));
    F lT3 = lnTc - F(6.907755278982137);
    F iT3 = F(1000) / m_min(m_max(T, F(10)), F(1e4));  // 1/T3 = exp(-lT3)
    k.rvLLTE = rovib_lte_of(lT3, iT3);
  }
  F st10 = m_sqrt(T * F(0.1));
  k.coA = F(4e-27) * (T * F(0.1)) * st10;
  k.coN = F(3e3) * st10;
  k.grT = F(4.65e-30) * m_exp(F(0.94) * lnT);
  k.grB = F(0.74) * m_exp(F(-0.068) * lnT);
  F poly = F(6.92e-1) + lT4 * (F(-5.86e-1) + lT4 * (F(8.16e-1) + lT4 * (F(-5.05e-1) +
           lT4 * (F(1.18e-1) + lT4 * (F(7.66e-3) + lT4 * F(-5.08e-3))))));
  k.nebT = F(3.68e-23) * m_exp(poly * F(LN10) - F(3.86) * invT4 - F(0.5) * lT4);
  k.nebX = F(0.38) - F(0.12) * lT4;
  if (flags & FL_NO_CIE) {
    k.cie = F(0);
  } else {
    k.cie = cie_of(c, lt);
  }
  return k;
}

// The temperature blocks at T1 = T + dT from those at T, for the forward-difference
// Jacobian's temperature column (dT ~ 1e-7 T).  A factor C exp(a ln T + b/T) moves by
// its logarithmic derivative, f(T1) = f(T) (1 + (a + b/T) dT/T); the factors that are
// sums of several such terms (the hot-gas electrons, Ly-alpha, the Gaunt factor, the H2
// LTE rate, CIE) and the products of stepped factors are evaluated at T1.  The neglected
// second-order term is ~((a + b/T) dT/T)^2 / 2 relative, far below the difference's
// own (a + b/T) dT/T, so the column agrees with the one from chem_T and cool_T at T1 to
// the forward difference's truncation error: 13 exponentials instead of 38.
template <class F>
TCG_BIG void temp_blocks_step(const CellC<F>& c, const ChemT<F>& b, const CoolT<F>& k, F T1, unsigned flags,
                              ChemT<F>& o, CoolT<F>& ok) {
  TCG_COUNT(temp_step);
  const F T = b.T, iT = b.invT;
  const F dT = T1 - T;
  const F u = dT * iT;   // dT / T
  const F ui = u * iT;   // dT / T^2
  // ---- chemistry block
  o.T = T1;
  o.lnT = b.lnT + u;
  o.sqT = b.sqT + b.sqT * (F(0.5) * u);
  o.invT = iT - iT * u;
  o.S = b.S + b.S * (F(1) - b.S) * (F(10.0 / 1.5e4) * dT);
  if (flags & FL_CONST_KGR) {
    o.kgr = b.kgr;
  } else {
    // k_gr = K s2 / D with s2 = sqrt(T/100), T2 = T/100, D = 1 + 0.4 s2 + 0.2 T2 + 0.08 T2^2
    F s2 = b.sqT * F(0.1), T2 = T * F(0.01);
    F D = F(1) + F(0.4) * s2 + F(0.2) * T2 + F(0.08) * T2 * T2;
    F dD = F(0.2) * s2 * iT + F(0.002) + F(0.0016) * T2;  // dD/dT
    o.kgr = b.kgr + b.kgr * (F(0.5) * u - dD * dT / D);
  }
  F lT4 = b.lnT - F(9.210340371976184);
  o.arr = b.arr + b.arr * ((F(-0.8163) - F(0.0416) * lT4) * u);
  F c3s = b.sqT * F(0.003162277660168379);
  o.kci = b.kci + b.kci * ((F(0.5) - F(0.5) * c3s / (F(1) + c3s)) * u + F(157809.1) * ui);
  o.kcdH = b.kcdH + b.kcdH * (F(0.5) * u + F(63593.0) * ui);
  o.kcdH2 = b.kcdH2 + b.kcdH2 * (F(4.1881) * u + F(54657.4) * ui -
                                 F(5.6881 * 6.761e-6) * dT / (F(1) + F(6.761e-6) * T));
  o.arrC = b.arrC - b.arrC * (F(0.6) * u);
  o.kCpH2 = b.kCpH2 - b.kCpH2 * (F(0.2) * u);
  o.xMH_T = b.xMH_T + b.xMH_T * (F(0.345) * u);
  F lt1 = o.lnT * F(0.43429448190325176);
  o.xe_hot = xe_hot_of(c, lt1);
  o.wdH3T = b.wdH3T + b.wdH3T * (F(WDH4) * u);
  o.wdHex = b.wdHex - F(WDH6) * u;
  o.wdC3T = b.wdC3T + b.wdC3T * (F(WDC4) * u);
  o.wdCex = b.wdCex - F(WDC6) * u;
  // ---- cooling block
  ok.fcA = k.fcA + k.fcA * (F(0.5) * u + F(1000.0) * ui);
  F T12 = T + F(1200.0);
  ok.fcB = k.fcB + k.fcB * (F(0.5) * u + F(18100.0) * dT / (T12 * T12));
  ok.eps_num = k.eps_num + (k.eps_num - F(5.22)) * (F(0.147) * u);
  F lT4_1 = o.lnT - F(9.210340371976184);
  ok.lyaE = lya_of(lT4_1, F(1e4) * o.invT);
  ok.ffrr = F(1.42e-27) * o.sqT * gff_of(lt1) + o.arr * F(KB) * T1 * (F(0.684) - F(0.0416) * lT4_1);
  ok.cpke = F(2.3e-6 / 53.0 * 100.0) * o.sqT * o.invT;
  F lT2 = b.lnT - F(4.605170185988092);
  ok.cpkH = k.cpkH + k.cpkH * ((F(0.1281) + F(0.0174) * lT2) * u);
  ok.cpb = k.cpb + k.cpb * (F(91.25) * ui);
  const F sO = F(-0.2622274154608984), sC = F(-0.22834652828762741);  // as in cool_T
  ok.ok10 = k.ok10 - k.ok10 * (sO * u);
  ok.ob1 = k.ob1 + k.ob1 * (F(227.7) * ui);
  ok.ob2 = k.ob2 + k.ob2 * (F(326.6) * ui);
  ok.ob21 = k.ob21 + k.ob21 * (F(326.6 - 227.7) * ui);
  ok.ck10 = k.ck10 - k.ck10 * (sC * u);
  ok.cb1 = k.cb1 + k.cb1 * (F(23.6) * ui);
  ok.cb2 = k.cb2 + k.cb2 * (F(62.4) * ui);
  ok.cb21 = k.cb21 + k.cb21 * (F(62.4 - 23.6) * ui);
  if (flags & FL_NO_ROVIB) {
    ok.rvLlow = k.rvLlow; ok.rvLLTE = k.rvLLTE;
  } else {
    // L_low = 10^poly(log10 T): d ln L_low / dT = poly'(log10 T) / T inside the clamp
    // [10, 1e4] K, zero outside
    if (b.lnT > F(2.302585092994046) && b.lnT < F(9.210340371976184)) {
      F x = b.lnT * F(0.43429448190325176);
      F dpoly = F(97.59) + x * (F(2 * -48.05) + x * (F(3 * 10.80) + x * F(4 * -0.9032)));
      ok.rvLlow = k.rvLlow + k.rvLlow * (dpoly * u);
    } else {
      ok.rvLlow = k.rvLlow;
    }
    F lnTc1 = m_min(m_max(o.lnT, F(2.302585092994046)), F(9.210340371976184));
    ok.rvLLTE = rovib_lte_of(lnTc1 - F(6.907755278982137), F(1000) / m_min(m_max(T1, F(10)), F(1e4)));
  }
  ok.coA = k.coA + k.coA * (F(1.5) * u);
  ok.coN = k.coN + k.coN * (F(0.5) * u);
  ok.grT = k.grT + k.grT * (F(0.94) * u);
  ok.grB = k.grB - k.grB * (F(0.068) * u);
  // nebular: ln f = ln 3.68e-23 + LN10 poly(lT4) - 3.86e4 / T - 0.5 lT4
  F dpn = F(-5.86e-1) + lT4 * (F(2 * 8.16e-1) + lT4 * (F(3 * -5.05e-1) + lT4 * (F(4 * 1.18e-1) +
          lT4 * (F(5 * 7.66e-3) + lT4 * F(6 * -5.08e-3)))));
  ok.nebT = k.nebT + k.nebT * ((F(LN10) * dpn - F(0.5)) * u + F(3.86e4) * ui);
  ok.nebX = k.nebX - F(0.12) * u;
  ok.cie = (flags & FL_NO_CIE) ? F(0) : cie_of(c, lt1);
}

// ------------------------------------------------------------------ C/O/e equilibrium (Secs. 3.2, 3.3)
template <class F> struct Equil {
  F xe, xCp, xCO, xC, xO, xOp, xMHp;
  F lpsi;  // ln psi at x_e, psi = G0 sqrt(T) / n_e + 50 (grain-charging parameter)
};

// Electron balance g(x_e) = x_e - a0 - w x_C+(x_e) = 0 (Eqs. e:xEL / e:xELhot blended by
// S(T), Eq. eq:C+_frac for x_C+), solved by Newton's method with the analytic derivative
// inside the bracket [a0, a0 + w x_C,tot] (bisection when a step leaves it), warm-started
// at `guess`, to a relative step of Prec<F>::root_tol (or after newton_max Newton steps).
template <class F> TCG_BIG Equil<F> equilibrium(const CellC<F>& c, const ChemT<F>& b, F xH2,
                                                                  F xHp, F guess, int newton_max = 100) {
  TCG_COUNT(equil);
  Equil<F> q;
  const F w = F(1) - b.S;
  q.xOp = c.xOtot * xHp;
  q.xMHp = F(2) * xH2 * c.xMH_pref * b.xMH_T;
  const F a0 = w * (xHp + q.xOp + q.xMHp) + b.S * (xHp + b.xe_hot);
  const F src = c.zpiC_rad + F(1040.0) * xH2 * c.xi + c.zcrC;  // zeta_pi,C + zeta_cr,C
  const F sink0 = src + b.kCpH2 * c.n * xH2;                     // + k_C+-H2 n_H2
  const F num = c.xCtot * src;
  const F Gs = c.G0 * b.sqT;
  const F agr0 = F(1e-14 * WDC0) * c.Zd;
  // x_C+(x), its derivative, ln psi(x) and d ln psi / dx
  auto xcp = [&](F x, F& dxcp, F& lp, F& dlp) -> F {
    F ne = x * c.n;
    F psi = Gs / m_max(ne, F(1e-30)) + F(50);
    lp = m_log(psi);
    F pa = m_exp(F(WDC2) * lp);
    F pb = b.wdC3T * m_exp(b.wdCex * lp);
    F D = F(1) + F(WDC1) * pa * (F(1) + pb);
    F invD = F(1) / D;
    F agr = agr0 * invD;
    F den = sink0 + (agr + b.arrC * x) * c.n;
    // dD/dx = dD/d ln psi  d ln psi/dx, with dD/d ln psi = C1 (C2 pa (1 + pb) + pa C5' pb)
    // and d ln psi/dx = -(psi - 50)/(psi x) when ne > floor; d agr/dx = -agr dD/dx / D
    dlp = (ne > F(1e-30)) ? -(psi - F(50)) / (psi * x) : F(0);
    F dDdx = F(WDC1) * (F(WDC2) * pa * (F(1) + pb) + pa * b.wdCex * pb) * dlp;
    F dagr = -agr * invD * dDdx;
    F invden = F(1) / den;
    F r = num * invden;
    dxcp = -r * invden * ((dagr + b.arrC) * c.n);
    return r;
  };
  F lo = a0, hi = a0 + w * c.xCtot;
  F xe;
  // the last evaluation of the iteration (point, x_C+, derivative, ln psi, d ln psi/dx)
  bool have_ev = false;
  F x_ev = F(0), r_ev = F(0), d_ev = F(0), lp_ev = F(0), dlp_ev = F(0);
  if (!(hi > lo) || !(num > F(0))) {
    xe = a0;
  } else {
    F x = (guess > lo && guess < hi) ? guess : hi;
    const F tol = F(Prec<F>::root_tol);
    xe = x;
    for (int it = 0; it < 100; ++it) {
      TCG_COUNT(equil_it);
      F d, lpx, dlpx;
      const F r = xcp(x, d, lpx, dlpx);
      x_ev = x; r_ev = r; d_ev = d; lp_ev = lpx; dlp_ev = dlpx;
      have_ev = true;
      F g = x - a0 - w * r;
      if (g == F(0)) { xe = x; break; }
      if (g > F(0)) hi = x; else lo = x;
      F gp = F(1) - w * d;
      F xn = x - g / gp;
      // a Newton step that lands on a bracket end is kept: near the root the bracket
      // collapses onto it, and bisecting there would only grind the bracket down
      const bool newton = (xn >= lo && xn <= hi);
      if (!newton) xn = F(0.5) * (lo + hi);
      F dx = m_abs(xn - x);
      x = xn;
      xe = x;
      if (dx <= tol * x || hi - lo <= tol * hi) break;
      // a caller whose guess is within ~1e-7 of the root (the Jacobian's perturbed
      // evaluations, started from the base point's root) stops after newton_max Newton
      // steps: one step from there is already converged to ~1e-14
      if (newton && it + 1 >= newton_max) break;
    }
  }
  q.xe = xe;
  // x_C+ and ln psi at the root (source() takes ln psi from here): the last evaluation
  // stepped to xe to first order when that step is small, |xe - x| <= 1e-6 xe.  That is
  // the solve's final Newton step: below the root tolerance when converged, so exact to
  // rounding, and ~1e-7 xe after the single capped step of the Jacobian's perturbed
  // evaluations, leaving ~1e-14 relative.  Otherwise (no iteration, or a solve stopped
  // far from its root) a fresh evaluation at xe.
  const F dxe = xe - x_ev;
  if (have_ev && m_abs(dxe) <= F(1e-6) * xe) {
    q.xCp = r_ev + d_ev * dxe;
    q.lpsi = lp_ev + dlp_ev * dxe;
  } else {
    F dd, dl;
    q.xCp = xcp(xe, dd, q.lpsi, dl);
  }
  F fr = m_max((c.xCtot > F(0)) ? q.xCp / c.xCtot : F(0), xHp);
  q.xCO = c.xCtot * F(2) * xH2 * (F(1) - fr) / (F(1) + c.rCO2);  // Eq. e:CO
  q.xC = c.xCtot - q.xCp - q.xCO;
  q.xO = c.xOtot - q.xCO - q.xOp;
  return q;
}

// ------------------------------------------------------------------ dust temperature (Eq. eq:dust_en)
// B T_d^2 (T_d^4 - T_cmb^4) = Gd + Cgd sqrt(T) (T - T_d): Newton inside a sign-change
// bracket, warm-started at `guess`.  Without a usable guess the start is the root of
// B T_d^6 = Gd + Cgd sqrt(T) T (the balance with the CMB and the T_d-dependence of the
// gas-dust term dropped), which is within a few Newton steps of the root; starting at
// the bracket midpoint instead would take ~70 linearly convergent steps in hot gas.
template <class F> TCG_FN F dust_T(const CellC<F>& c, F T, F sqT, F guess) {
  if (!(c.Zd > F(0))) return T;
  TCG_COUNT(dust);
  F C = c.Cgd * sqT;
  F lo = m_min(T, c.Tc);
  F hi = m_max(m_max(T, F(1.2) * c.Tc), c.Td_hi);
  F y = guess;
  if (!(y > lo && y < hi)) {
    y = m_exp(m_log((c.Gd + C * T) / c.Bd) * F(1.0 / 6.0));
    if (!(y > lo && y < hi)) y = F(0.5) * (lo + hi);
  }
  const F tol = F(Prec<F>::root_tol);
  for (int it = 0; it < 100; ++it) {
    TCG_COUNT(dust_it);
    F y2 = y * y;
    F h = c.Bd * y2 * (y2 * y2 - c.Tc4) - c.Gd - C * (T - y);
    if (h > F(0)) hi = y; else lo = y;
    F dh = c.Bd * y * (F(6) * y2 * y2 - F(2) * c.Tc4) + C;
    F yn = y - h / dh;
    if (!(yn >= lo && yn <= hi)) yn = F(0.5) * (lo + hi);  // bracket ends allowed, as above
    F dy = m_abs(yn - y);
    y = yn;
    if (dy <= tol * y || hi - lo <= tol * hi) break;
  }
  return y;
}

// ------------------------------------------------------------------ hydrogen rates at (T, x, x_e)
template <class F> struct HRate {
  F kn;    // k_gr n
  F DH2;   // 1.65 zeta_cr,H2 + zeta_pd + zeta_pi,H2 + zeta_cd
  F I;     // zeta_pi,H + zeta_cr,H + zeta_ci
  F Rr;    // alpha_rr n_e + alpha_gr n
};

// xH is the atomic fraction 1 - 2 x_H2 - x_H+ (Sec. 3.1.3), passed in so that the
// mixed-precision path can form it in FP64 and hand the FP32 rates an accurate value
// when x_H+ -> 1 or x_H2 -> 1/2.
template <class F> TCG_FN HRate<F> h_rates(const CellC<F>& c, const ChemT<F>& b, F xH2, F xH,
                                                               F xe, F lpsi) {
  HRate<F> r;
  F zcrH2 = F(2) * c.xi * (F(2.3) * xH2 + F(1.5) * xH);        // Eq. eq:H2_cr
  F zcd = c.n * (b.kcdH * xH + b.kcdH2 * xH2);
  F ne = xe * c.n;
  F agrH = F(1e-14 * WDH0) * c.Zd /
           (F(1) + F(WDH1) * m_exp(F(WDH2) * lpsi) * (F(1) + b.wdH3T * m_exp(b.wdHex * lpsi)));
  r.kn = b.kgr * c.n;
  r.DH2 = F(1.65) * zcrH2 + c.zpd + c.zpiH2 + zcd;
  r.I = c.zpiH + F(0.5) * zcrH2 + b.kci * ne;
  r.Rr = b.arr * ne + agrH * c.n;
  return r;
}

template <class F> TCG_FN F log_psi(const CellC<F>& c, const ChemT<F>& b, F xe) {
  return m_log(c.G0 * b.sqT / m_max(xe * c.n, F(1e-30)) + F(50));
}

// ------------------------------------------------------------------ net source terms
template <class F> struct Src {
  F H;          // n Gamma - n^2 Lambda [erg cm^-3 s^-1]
  F CH2, CHp;   // Eqs. e:HH, e:HII [s^-1]
  F Td;
  F G, L;       // heating per H [erg s^-1] and cooling per n_H^2 [erg cm^3 s^-1]
  F form, dest; // k_gr n x_H and D_H2 x_H2: the two sides of Eq. e:HH
  F ion, rec;   // I x_H and R x_H+: the two sides of Eq. e:HII
};

// Heating (Eq. e:heating) and cooling (Eq. eq:cooling_fnct) at (T, x_H2, x_H+, q) with
// the atomic fraction xH given.  Td_fixed > 0 freezes the dust temperature; otherwise it
// is solved from Td_guess.
template <class F> TCG_BIG Src<F> source(const CellC<F>& c, const ChemT<F>& b, const CoolT<F>& k,
                                                            F xH2, F xHp, F xH, const Equil<F>& q, F Td_fixed,
                                                            F Td_guess) {
  TCG_COUNT(source);
  Src<F> s;
  const F n = c.n;
  const F xe = q.xe;
  const F lp = q.lpsi;  // log_psi(c, b, xe) from the equilibrium solve (to ~1e-14 relative)
  const HRate<F> r = h_rates(c, b, xH2, xH, xe, lp);
  s.form = r.kn * xH;
  s.dest = r.DH2 * xH2;
  s.ion = r.I * xH;
  s.rec = r.Rr * xHp;
  s.CH2 = s.form - s.dest;
  s.CHp = s.ion - s.rec;
  // --- heating per H
  F eps = k.eps_num / (F(1) + F(0.04996) * m_exp(F(0.431) * lp) * (F(1) + F(0.00430) * m_exp(F(0.692) * lp)));
  F qH = (F(7.5) + F(24.5) * m_sqrt(xe / (xe + F(0.07)))) * F(EV);
  F dcol = n * (xH * k.fcA + xH2 * k.fcB);
  F fcol = dcol / (dcol + F(2e-7) + c.zpd);
  F G = F(1e-26) * c.G0 * eps * c.Zd                                  // photoelectric
      + c.xi * (xH * qH + F(2) * xH2 * c.qH2)                           // cosmic rays
      + xH * F(3.4 * EV) * c.zpiH + xH2 * F(4.4 * EV) * c.zpiH2         // photoionisation
      + r.kn * xH * (F(0.2 * EV) + F(4.2 * EV) * fcol)                  // H2 formation
      + c.zpd * xH2 * (F(16.0 * EV) * fcol + F(0.4 * EV));             // UV pumping + dissociation
  // --- cooling per n^2
  F Lhyd = xH * xe * (k.lyaE + F(13.6 * EV) * b.kci)                  // Ly-alpha + coll. ionisation
         + F(4.48 * EV) * xH2 * (xH * b.kcdH + xH2 * b.kcdH2)          // coll. dissociation
         + k.ffrr * xe * xHp;                                           // free-free + recombination
  {
    F nL = n * k.rvLlow;                                                // H2 ro-vibrational
    F den = nL + k.rvLLTE;
    // harmonic combination L_LTE n L_low / (n L_low + L_LTE); in FP32's exponent range
    // the product of the two rates (~1e-22 x 1e-24) underflows, so the ratio is taken
    // first there.
    F Lrv;
    if constexpr (Prec<F>::fp32_range) Lrv = k.rvLLTE * (nL / den);
    else Lrv = k.rvLLTE * nL / den;
    Lhyd += (den > F(0)) ? xH2 * Lrv / n : F(0);
  }
  F Lmet;
  {
    // C+ two-level
    F C10 = n * (k.cpke * xe + k.cpkH * (xH + F(0.5) * xH2));
    F C01 = C10 * k.cpb;
    // (energies in K; k_B and 1/n applied once at the end, which keeps the partial
    // sums far above FP32's smallest normal number)
    F lines = q.xCp * (C01 / (F(2.3e-6) + C10 + C01)) * F(2.3e-6 * 91.25);
    // O and C three-level atoms, H and H2 collisions (H2 at half the H rate).  The level
    // populations relative to the ground state are r1 = p1/det and r2 = p2/det, and the
    // cooling per atom (r1 A1 E1 + r2 (A20 E2 + A21 E21)) / (1 + r1 + r2) is taken as
    // (p1 A1 E1 + p2 (...)) / (det + p1 + p2), one quotient instead of three.
    F coll = n * (xH + F(0.5) * xH2);
    {
      F C10o = k.ok10 * coll;
      F C01o = C10o * k.ob1, C02o = C10o * k.ob2, C12o = C10o * k.ob21;
      F a11 = F(8.91e-5) + C10o + C12o;
      F bb = F(1.75e-5) + C10o;
      F a22 = F(1.34e-10) + F(1.75e-5) + F(2) * C10o;
      F det = a11 * a22 - bb * C12o;
      F p1 = C01o * a22 + bb * C02o;
      F p2 = a11 * C02o + C12o * C01o;
      lines += q.xO * (p1 * F(8.91e-5 * 227.7) + p2 * F(1.34e-10 * 326.6 + 1.75e-5 * (326.6 - 227.7))) /
               (det + p1 + p2);
    }
    {
      F C10c = k.ck10 * coll;
      F C01c = C10c * k.cb1, C02c = C10c * k.cb2, C12c = C10c * k.cb21;
      F a11 = F(7.93e-8) + C10c + C12c;
      F bb = F(2.65e-7) + C10c;
      F a22 = F(2.0e-14) + F(2.65e-7) + F(2) * C10c;
      F det = a11 * a22 - bb * C12c;
      F p1 = C01c * a22 + bb * C02c;
      F p2 = a11 * C02c + C12c * C01c;
      lines += q.xC * (p1 * F(7.93e-8 * 23.6) + p2 * F(2.0e-14 * 62.4 + 2.65e-7 * (62.4 - 23.6))) /
               (det + p1 + p2);
    }
    Lmet = lines * F(KB) / n;
    // CO (stand-in with LVG-like trapping)
    Lmet += q.xCO * k.coA / (F(1) + n / k.coN + q.xCO * c.NtX * F(1e-17));
    // grain-assisted recombination
    Lmet += k.grT * m_exp(k.grB * lp) * xe * c.Zd;
    // nebular lines (Eq. e:Lambda_neb)
    F ne2 = xe * n * F(0.01);
    Lmet += c.Zg * xe * xHp * k.nebT / (F(1) + F(0.12) * m_exp(k.nebX * m_log(ne2)));
    // gas-dust (Eq. eq:gas-dust)
    s.Td = (Td_fixed > F(0)) ? Td_fixed : dust_T(c, b.T, b.sqT, Td_guess);
    Lmet += F(3.2e-34) * b.sqT * (b.T - s.Td) * c.Zd;
  }
  F L = Lhyd + (F(1) - b.S) * Lmet + b.S * k.cie;
  s.G = G;
  s.L = L;
  s.H = n * G - n * n * L;
  return s;
}

}  // namespace tcg
