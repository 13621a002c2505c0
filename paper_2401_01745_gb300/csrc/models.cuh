// Ionic models in Hodgkin-Huxley form for the CUDA path (Sec. 2, Eq. monodomain).
//
// Each model exposes, per node and templated on the arithmetic type R
// (double for the FP64 path, float for the mixed path):
//   gating_each(V, zE, zS, cb)    : calls cb(k, Lambda_k, z_inf_k) for every gate k
//                                   as soon as both are known, so that a caller
//                                   can consume a gate while the next is computed;
//                                   g_E = Lambda_E (zE - z_inf).  Gates in
//                                   alpha/beta form use Lambda = -(alpha+beta),
//                                   z_inf = alpha/(alpha+beta); tau-form gates use
//                                   Lambda = -1/tau.
//   gating(V, zE, zS, lam, zinf)  : the same into arrays.
//   currents(V, zE, zS, Iion, gS) : total ionic current (uA/cm^2 at 1 uF/cm^2) and
//                                   the right-hand side g_S of the non-gating
//                                   variables (Eq. mono_in_FSE).
// The exponential (Rush-Larsen) step itself is applied by the stage kernels.
// Divisions by constants are written as multiplications by the reciprocal
// constant (folded at compile time): one rounding instead of a division.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace emrkc {

template <typename R> struct Math;

template <> struct Math<double> {
  static __device__ __forceinline__ double ex(double x) { return exp(x); }
  static __device__ __forceinline__ double em1(double x) { return expm1(x); }
  static __device__ __forceinline__ double ln(double x) { return log(x); }
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
  static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
  // e^{s (x - c)} for constants c, s, evaluated as written
  static __device__ __forceinline__ double ex_aff(double x, double c, double s) { return exp((x - c) * s); }
  // x / (e^x - 1) with the removable singularity at 0 (1 - x/2 for |x| < 1e-7)
  static __device__ __forceinline__ double x_em1(double x) {
    return fabs(x) < 1e-7 ? 1.0 - 0.5 * x : x / expm1(x);
  }
};

template <> struct Math<float> {
  static __device__ __forceinline__ float ex(float x) { return __expf(x); }
  // e^x - 1: Taylor polynomial through x^4 for |x| < 1/32 (relative truncation
  // error below x^4/120 < 1e-8), e^x - 1 otherwise (|e^x - 1| > 0.03 there).
  static __device__ __forceinline__ float em1(float x) {
    if (fabsf(x) < 0.03125f) return x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f))));
    return __expf(x) - 1.0f;
  }
  static __device__ __forceinline__ float ln(float x) { return __logf(x); }
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
  // e^{s (x - c)} for constants c, s as 2^(x s log2(e) - c s log2(e)): one
  // fused multiply-add with constants folded at compile time and the hardware
  // base-2 exponential (ex2.approx, relative error ~2^-22)
  static __device__ __forceinline__ float ex_aff(float x, double c, double s) {
    constexpr double kLog2e = 1.4426950408889634074;
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaf(x, (float)(s * kLog2e), (float)(-c * s * kLog2e))));
    return r;
  }
  static __device__ __forceinline__ float x_em1(float x) {
    return fabsf(x) < 1e-4f ? 1.0f - 0.5f * x : __fdividef(x, em1(x));
  }
};

// ---------------------------------------------------------------------------
// Pure diffusion: V only.
template <typename R> struct ModelNone {
  static constexpr int NE = 0, NS = 0;
  template <class CB>
  static __device__ __forceinline__ void gating_each(R, const R*, const R*, CB&&) {}
  static __device__ __forceinline__ void gating(R, const R*, const R*, R*, R*) {}
  static __device__ __forceinline__ void currents(R, const R*, const R*, R& I, R*) { I = R(0); }
  static __host__ __device__ constexpr double rest(int) { return 0.0; }
};

// ---------------------------------------------------------------------------
// Linear passive test model: I_ion = g_p V, one gate w with constant rates,
// one auxiliary c with g_S = -k_c c.  All three components are decoupled.
template <typename R> struct ModelPassive {
  static constexpr int NE = 1, NS = 1;
  template <class CB>
  static __device__ __forceinline__ void gating_each(R, const R*, const R*, CB&& cb) {
    cb(0, -(R(20) + R(30)), R(20) / (R(20) + R(30)));
  }
  static __device__ __forceinline__ void gating(R V, const R* zE, const R* zS, R* lam, R* zinf) {
    gating_each(V, zE, zS, [&](int k, R l, R zi) {
      lam[k] = l;
      zinf[k] = zi;
    });
  }
  static __device__ __forceinline__ void currents(R V, const R*, const R* zS, R& I, R* gS) {
    I = R(0.5) * V;
    gS[0] = -R(2) * zS[0];
  }
  static __host__ __device__ constexpr double rest(int k) {
    return k == 0 ? 0.0 : 1.0;
  }
};

// ---------------------------------------------------------------------------
// Hodgkin-Huxley 1952 (modern sign convention, V_rest = -75 mV).
// Rates in v = V - V_rest; reversal potentials V_rest + 115, V_rest - 12,
// V_rest + 10.613; conductances 120, 36, 0.3 mS/cm^2.
template <typename R> struct ModelHH {
  static constexpr int NE = 3, NS = 0;
  using M = Math<R>;
  static __device__ __forceinline__ void rates(R V, R* a, R* b) {
    const R v = V - R(-75.0);
    a[0] = M::x_em1((R(25.0) - v) * R(1.0 / 10.0));      // alpha_m = 0.1(25-v)/(e^{(25-v)/10}-1)
    b[0] = R(4.0) * M::ex(-v * R(1.0 / 18.0));            // beta_m
    a[1] = R(0.07) * M::ex(-v * R(1.0 / 20.0));           // alpha_h
    b[1] = R(1.0) / (M::ex((R(30.0) - v) * R(1.0 / 10.0)) + R(1.0));  // beta_h
    a[2] = R(0.1) * M::x_em1((R(10.0) - v) * R(1.0 / 10.0));  // alpha_n = 0.01(10-v)/(e^{(10-v)/10}-1)
    b[2] = R(0.125) * M::ex(-v * R(1.0 / 80.0));          // beta_n
  }
  template <class CB>
  static __device__ __forceinline__ void gating_each(R V, const R*, const R*, CB&& cb) {
    R a[3], b[3];
    rates(V, a, b);
#pragma unroll
    for (int k = 0; k < 3; ++k) cb(k, -(a[k] + b[k]), a[k] / (a[k] + b[k]));
  }
  static __device__ __forceinline__ void gating(R V, const R* zE, const R* zS, R* lam, R* zinf) {
    gating_each(V, zE, zS, [&](int k, R l, R zi) {
      lam[k] = l;
      zinf[k] = zi;
    });
  }
  static __device__ __forceinline__ void currents(R V, const R* zE, const R*, R& I, R*) {
    const R m = zE[0], h = zE[1], n = zE[2];
    const R n2 = n * n;
    I = R(120.0) * (m * m * m) * h * (V - R(-75.0 + 115.0)) +
        R(36.0) * (n2 * n2) * (V - R(-75.0 - 12.0)) + R(0.3) * (V - R(-75.0 + 10.613));
  }
};

// ---------------------------------------------------------------------------
// ten Tusscher & Panfilov 2006, epicardial cell.
// Gates z_E: m h j xr1 xr2 xs r s d f f2 fCass; z_S: Rbar Ki Nai Cai CaSR CaSS.
// Currents in pA/pF, time in ms, concentrations in mM; free calcium is the
// state and fast buffering enters through beta = 1/(1 + B K/(c + K)^2).
template <typename R> struct ModelTTP06 {
  static constexpr int NE = 12, NS = 6;
  using M = Math<R>;
  // physical constants (R in mJ/(K mol), F in C/mol), cell geometry
  static constexpr double Rgas = 8314.472, Temp = 310.0, Far = 96485.3415;
  static constexpr double Cap = 0.185, Vc = 0.016404, Vsr = 0.001094, Vss = 0.00005468;
  static constexpr double Ko = 5.4, Nao = 140.0, Cao = 2.0;

  static __device__ __forceinline__ R sig(R x) { return R(1) / (R(1) + M::ex(x)); }
  // 1 / (1 + e^{s (V - c)})
  static __device__ __forceinline__ R sg(R V, double c, double s) { return R(1) / (R(1) + M::ex_aff(V, c, s)); }

  template <class CB>
  static __device__ __forceinline__ void gating_each(R V, const R*, const R* zS, CB&& cb) {
    const R CaSS = zS[5];
    // I_Na gates
    {
      const R s = sg(V, -56.86, -(1.0 / 9.03));
      const R am = sg(V, -60.0, -(1.0 / 5.0));
      const R bm = R(0.1) * sg(V, -35.0, 1.0 / 5.0) + R(0.10) * sg(V, 50.0, 1.0 / 200.0);
      cb(0, -R(1) / (am * bm), s * s);
    }
    const R hs = sg(V, -71.55, 1.0 / 7.43);
    if (V >= R(-40.0)) {
      const R bh = R(0.77) / (R(0.13) * (R(1) + M::ex_aff(V, -10.66, -(1.0 / 11.1))));
      cb(1, -bh, hs * hs);  // alpha_h = 0
      const R bj = R(0.6) * M::ex_aff(V, 0.0, 0.057) / (R(1) + M::ex_aff(V, -32.0, -0.1));
      cb(2, -bj, hs * hs);  // alpha_j = 0
    } else {
      const R ah = R(0.057) * M::ex_aff(V, -80.0, -(1.0 / 6.8));
      const R bh = R(2.7) * M::ex_aff(V, 0.0, 0.079) + R(3.1e5) * M::ex_aff(V, 0.0, 0.3485);
      cb(1, -(ah + bh), hs * hs);
      const R aj = (R(-2.5428e4) * M::ex_aff(V, 0.0, 0.2444) - R(6.948e-6) * M::ex_aff(V, 0.0, -0.04391)) *
                   (V + R(37.78)) / (R(1) + M::ex_aff(V, -79.23, 0.311));
      const R bj = R(0.02424) * M::ex_aff(V, 0.0, -0.01052) / (R(1) + M::ex_aff(V, -40.14, -0.1378));
      cb(2, -(aj + bj), hs * hs);
    }
    // I_Kr gates
    cb(3, -R(1) / ((R(450.0) * sg(V, -45.0, -(1.0 / 10.0))) * (R(6.0) * sg(V, -30.0, 1.0 / 11.5))),
       sg(V, -26.0, -(1.0 / 7.0)));
    cb(4, -R(1) / ((R(3.0) * sg(V, -60.0, -(1.0 / 20.0))) * (R(1.12) * sg(V, 60.0, 1.0 / 20.0))),
       sg(V, -88.0, 1.0 / 24.0));
    // I_Ks gate
    cb(5,
       -R(1) / ((R(1400.0) / M::sq(R(1) + M::ex_aff(V, 5.0, -(1.0 / 6.0)))) * sg(V, 35.0, 1.0 / 15.0) + R(80.0)),
       sg(V, -5.0, -(1.0 / 14.0)));
    // I_to gates (epicardial s)
    {
      const R d40 = V + R(40.0);
      cb(6, -R(1) / (R(9.5) * M::ex(-(d40 * d40) * R(1.0 / 1800.0)) + R(0.8)), sg(V, 20.0, -(1.0 / 6.0)));
    }
    {
      const R d45 = V + R(45.0);
      cb(7, -R(1) / (R(85.0) * M::ex(-(d45 * d45) * R(1.0 / 320.0)) + R(5.0) * sg(V, 20.0, 1.0 / 5.0) + R(3.0)),
         sg(V, -20.0, 1.0 / 5.0));
    }
    // I_CaL gates
    cb(8,
       -R(1) / ((R(1.4) * sg(V, -35.0, -(1.0 / 13.0)) + R(0.25)) * (R(1.4) * sg(V, -5.0, 1.0 / 5.0)) +
                sg(V, 50.0, -(1.0 / 20.0))),
       sg(V, -8.0, -(1.0 / 7.5)));
    {
      const R d27 = V + R(27.0);
      cb(9,
         -R(1) / (R(1102.5) * M::ex(-(d27 * d27) * R(1.0 / 225.0)) + R(200.0) * sg(V, 13.0, -(1.0 / 10.0)) +
                  R(180.0) * sg(V, -30.0, 1.0 / 10.0) + R(20.0)),
         sg(V, -20.0, 1.0 / 7.0));
    }
    {
      const R d25 = V + R(25.0);
      cb(10,
         -R(1) / (R(600.0) * M::ex(-(d25 * d25) * R(1.0 / 170.0)) + R(31.0) * sg(V, 25.0, -(1.0 / 10.0)) +
                  R(16.0) * sg(V, -30.0, 1.0 / 10.0)),
         R(0.67) * sg(V, -35.0, 1.0 / 7.0) + R(0.33));
    }
    {
      const R c = CaSS * R(1.0 / 0.05);
      const R q = R(1) + c * c;
      cb(11, -R(1) / (R(80.0) / q + R(2.0)), R(0.6) / q + R(0.4));
    }
  }
  static __device__ __forceinline__ void gating(R V, const R* zE, const R* zS, R* lam, R* zinf) {
    gating_each(V, zE, zS, [&](int k, R l, R zi) {
      lam[k] = l;
      zinf[k] = zi;
    });
  }

  static __device__ __forceinline__ void currents(R V, const R* zE, const R* zS, R& Iion, R* gS) {
    const R m = zE[0], h = zE[1], j = zE[2], xr1 = zE[3], xr2 = zE[4], xs = zE[5];
    const R r = zE[6], s = zE[7], d = zE[8], f = zE[9], f2 = zE[10], fcass = zE[11];
    const R Rbar = zS[0], Ki = zS[1], Nai = zS[2], Cai = zS[3], CaSR = zS[4], CaSS = zS[5];
    const R RTF = R(Rgas * Temp / Far);
    const R iRTF = R(1) / RTF;
    const R E_K = RTF * M::ln(R(Ko) / Ki);
    const R E_Na = RTF * M::ln(R(Nao) / Nai);
    const R E_Ks = RTF * M::ln((R(Ko) + R(0.03) * R(Nao)) / (Ki + R(0.03) * Nai));
    const R E_Ca = R(0.5) * RTF * M::ln(R(Cao) / Cai);
    const R sqko = M::sq(R(Ko) * R(1.0 / 5.4));
    const R VK = V - E_K;
    const R aK1 = R(0.1) / (R(1) + M::ex_aff(VK, 200.0, 0.06));
    const R bK1 = (R(3.0) * M::ex_aff(VK, -100.0, 0.0002) + M::ex_aff(VK, 10.0, 0.1)) /
                  (R(1) + M::ex_aff(VK, 0.0, -0.5));
    const R I_K1 = R(5.405) * sqko * (aK1 / (aK1 + bK1)) * VK;
    const R I_to = R(0.294) * r * s * VK;
    const R I_Kr = R(0.153) * sqko * xr1 * xr2 * VK;
    const R I_Ks = R(0.392) * xs * xs * (V - E_Ks);
    const R I_Na = R(14.838) * (m * m * m) * h * j * (V - E_Na);
    const R I_bNa = R(0.00029) * (V - E_Na);
    const R u = R(2.0) * (V - R(15.0)) * iRTF;
    const R I_CaL = R(3.980e-5) * d * f * f2 * fcass * R(2.0 * Far) * M::x_em1(u) *
                    (R(0.25) * CaSS * M::ex(u) - R(Cao));
    const R I_bCa = R(0.000592) * (V - E_Ca);
    const R e1 = M::ex(R(0.35) * V * iRTF);
    const R e2 = M::ex(R(0.35 - 1.0) * V * iRTF);
    const R Nai3 = Nai * Nai * Nai;
    const R I_NaCa = R(1000.0) * (e1 * Nai3 * R(Cao) - e2 * R(Nao * Nao * Nao) * Cai * R(2.5)) /
                     (R((87.5 * 87.5 * 87.5 + Nao * Nao * Nao) * (1.38 + Cao)) * (R(1) + R(0.1) * e2));
    const R I_NaK = R(2.724) * R(Ko / (Ko + 1.0)) * Nai / (Nai + R(40.0)) /
                    (R(1) + R(0.1245) * M::ex(R(-0.1) * V * iRTF) + R(0.0353) * M::ex(-V * iRTF));
    const R I_pCa = R(0.1238) * Cai / (R(0.0005) + Cai);
    const R I_pK = R(0.0146) * VK / (R(1) + M::ex_aff(V, 25.0, -(1.0 / 5.98)));
    Iion = I_Kr + I_Ks + I_K1 + I_to + I_Na + I_bNa + I_CaL + I_bCa + I_NaK + I_NaCa + I_pCa + I_pK;

    // calcium dynamics
    const R rs = R(1) + (R(1.5) / CaSR) * (R(1.5) / CaSR);
    const R kcasr = R(2.5) - R(2.5 - 1.0) / rs;
    const R k1 = R(0.15) / kcasr;
    const R k2 = R(0.045) * kcasr;
    const R CaSS2 = CaSS * CaSS;
    const R O = k1 * CaSS2 * Rbar / (R(0.060) + k1 * CaSS2);
    const R I_rel = R(0.102) * O * (CaSR - CaSS);
    const R kc = R(0.00025) / Cai;
    const R I_up = R(0.006375) / (R(1) + kc * kc);
    const R I_leak = R(0.00036) * (CaSR - Cai);
    const R I_xfer = R(0.0038) * (CaSS - Cai);
    const R ci = Cai + R(0.001), csr = CaSR + R(0.3), css = CaSS + R(0.00025);
    const R b_c = R(1) / (R(1) + R(0.2 * 0.001) / (ci * ci));
    const R b_sr = R(1) / (R(1) + R(10.0 * 0.3) / (csr * csr));
    const R b_ss = R(1) / (R(1) + R(0.4 * 0.00025) / (css * css));
    const R capF = R(Cap / (Vc * Far));
    gS[0] = -k2 * CaSS * Rbar + R(0.005) * (R(1) - Rbar);
    gS[1] = -(I_K1 + I_to + I_Kr + I_Ks - R(2) * I_NaK + I_pK) * capF;
    gS[2] = -(I_Na + I_bNa + R(3) * I_NaK + R(3) * I_NaCa) * capF;
    gS[3] = b_c * ((I_leak - I_up) * R(Vsr / Vc) + I_xfer - (I_bCa + I_pCa - R(2) * I_NaCa) * R(0.5) * capF);
    gS[4] = b_sr * (I_up - I_rel - I_leak);
    gS[5] = b_ss * (-I_CaL * R(Cap / (2.0 * Vss * Far)) + I_rel * R(Vsr / Vss) - I_xfer * R(Vc / Vss));
  }
};

}  // namespace emrkc
