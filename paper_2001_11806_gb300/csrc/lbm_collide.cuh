// Per-cell collision operators, computed in registers on shifted populations
// h_q = f_q - w_q (so rho - 1 = sum h is accurate in FP32).
//
//   Eq. density: rho = sum f, u = (sum c f + F/2) / rho_0 (rho_0 = rho, or 1
//     for the incompressible variant of Sec. III-A; F/2 is the Guo half force).
//   Eq. discrete_eq (second order):
//     h^eq_q = w_q [ (rho - 1) + rho_0 (3 c.u + 9/2 (c.u)^2 - 3/2 u.u) ].
//   Guo source: G_q = w_q [3 (c_q - u).F + 9 (c_q.u)(c_q.F)].
//   With g = h - h^eq + G/2 every operator is h* = h + G - R g:
//     SRT  (Eq. bgk):  R = omega I;
//     TRT  (Sec. III-C): R = omega_e on the even part, omega_o on the odd part
//          of each opposite pair;
//     MRT  (Eq. mrt):  R = M^-1 S M = W M^T D^-1 S M for the w-orthogonal
//          basis of lbm_mrt.cuh.
//   The cumulant operator (Sec. III-B) is in lbm_cumulant.cuh.
#pragma once
#include <utility>

#include "lbm_lattice.cuh"
#include "lbm_mrt.cuh"

namespace lbm {

// OP_SRT_LES / OP_TRT_LES: SRT / TRT with the Smagorinsky model compiled in;
// OP_KBC: the entropic KBC operator; OP_MRT3: MRT whose moments of order
// >= 3 share one rate (see collide_mrt3)
enum Op : int {
  OP_SRT = 0, OP_TRT = 1, OP_MRT = 2, OP_CUM = 3, OP_SRT_LES = 4, OP_TRT_LES = 5, OP_KBC = 6, OP_MRT3 = 7
};

// Runtime parameters of a sweep, passed by value to the kernel.
struct CollideParams {
  float om[6];          // FP32 copies of the rates (see rates_d for FP64)
  double om_d[6];
  float mrt_s[27];      // s_k / D_k per MRT moment, FP32
  double mrt_s_d[27];   // s_k / D_k per MRT moment, FP64
  double F[3];          // body force
  int has_force;
  int incompressible;
  double u_wall[3];
  double rho_out;
  // Smagorinsky model (SRT/TRT): 18 C_S^2, tau_0 = 1/omega_0, magic Lambda
  int smag;
  int smag_magic;
  double smag_18cs2, smag_tau0, smag_lambda;
};

template <class T> __device__ __forceinline__ T rate(const CollideParams& p, int i);
template <> __device__ __forceinline__ float rate<float>(const CollideParams& p, int i) { return p.om[i]; }
template <> __device__ __forceinline__ double rate<double>(const CollideParams& p, int i) { return p.om_d[i]; }
template <class T> __device__ __forceinline__ T mrt_factor(const CollideParams& p, int k);
template <> __device__ __forceinline__ float mrt_factor<float>(const CollideParams& p, int k) { return p.mrt_s[k]; }
template <> __device__ __forceinline__ double mrt_factor<double>(const CollideParams& p, int k) { return p.mrt_s_d[k]; }

template <class L, class T>
struct Macro {
  T drho;   // rho - 1
  T rho0;   // rho (compressible) or 1
  T u[3];
  T F[3];
};

template <class L, class T>
__device__ __forceinline__ Macro<L, T> macro_from_h(const T (&h)[L::Q], const CollideParams& p) {
  Macro<L, T> m;
  T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    drho += h[q];
    if (L::cx(q) == 1) jx += h[q];
    if (L::cx(q) == -1) jx -= h[q];
    if (L::cy(q) == 1) jy += h[q];
    if (L::cy(q) == -1) jy -= h[q];
    if (L::cz(q) == 1) jz += h[q];
    if (L::cz(q) == -1) jz -= h[q];
  }
  m.F[0] = m.F[1] = m.F[2] = T(0);
  if (p.has_force) {
    m.F[0] = T(p.F[0]); m.F[1] = T(p.F[1]); m.F[2] = T(p.F[2]);
    jx += T(0.5) * m.F[0]; jy += T(0.5) * m.F[1]; jz += T(0.5) * m.F[2];
  }
  m.drho = drho;
  m.rho0 = p.incompressible ? T(1) : T(1) + drho;
  T inv = T(1) / m.rho0;
  m.u[0] = jx * inv; m.u[1] = jy * inv; m.u[2] = L::D == 3 ? jz * inv : T(0);
  return m;
}

// c_q . v for a small vector v.
template <class L, class T>
__device__ __forceinline__ T cdot(int q, const T (&v)[3]) {
  T r = T(0);
  if (L::cx(q) == 1) r += v[0];
  if (L::cx(q) == -1) r -= v[0];
  if (L::cy(q) == 1) r += v[1];
  if (L::cy(q) == -1) r -= v[1];
  if (L::D == 3) {
    if (L::cz(q) == 1) r += v[2];
    if (L::cz(q) == -1) r -= v[2];
  }
  return r;
}

// Even and odd parts of h^eq for direction q (q and opp(q) share them).
template <class L, class T>
__device__ __forceinline__ void heq_parts(int q, const Macro<L, T>& m, T usq15, T& even, T& odd) {
  const T w = T(L::w(q));
  const T cu = cdot<L, T>(q, m.u);
  even = w * (m.drho + m.rho0 * (T(4.5) * cu * cu - usq15));
  odd = w * m.rho0 * T(3) * cu;
}

// Guo source split into even and odd parts for direction q.
template <class L, class T>
__device__ __forceinline__ void guo_parts(int q, const Macro<L, T>& m, T uF3, T& even, T& odd) {
  const T w = T(L::w(q));
  const T cF = cdot<L, T>(q, m.F);
  const T cu = cdot<L, T>(q, m.u);
  even = w * (T(9) * cu * cF - uF3);
  odd = w * T(3) * cF;
}

// ---------------------------------------------------------------- SRT / TRT
// Pair form.  For each opposite pair (q, qbar) let s = h_q + h_qbar and
// d = h_q - h_qbar (h = f - w); then (TRT, Sec. III-C)
//   h*_q    = A + B,  h*_qbar = A - B,
//   A = (1 - omega_e) s/2 + omega_e h^eq+_q + (1 - omega_e/2) G+_q,
//   B = (1 - omega_o) d/2 + omega_o h^eq-_q + (1 - omega_o/2) G-_q,
//   h^eq+_q = w_q ((rho - 1) + rho_0 (9/2 (c.u)^2 - 3/2 u.u)),
//   h^eq-_q = 3 w_q rho_0 c.u,
// and SRT (Eq. bgk) is omega_o = omega_e.  rho and j come from the same s and
// d.  With unshifted storage (DH = false) the registers hold f: the pair sums
// are shifted by 2 w_q on the fly and w_q is added back once to each result,
// so the arithmetic, and its rounding, is that of the shifted form.
template <class T>
__device__ __forceinline__ void acc_signed(T& acc, bool& init, int sign, T x) {
  if (sign == 0) return;
  if (!init) { acc = sign > 0 ? x : -x; init = true; }
  else acc = sign > 0 ? acc + x : acc - x;
}

template <class L, class T, int OP, bool DH>
__device__ __forceinline__ void collide_pairs(T (&v)[L::Q], const CollideParams& p) {
  constexpr int NP = (L::Q - 1) / 2;
  T s[NP], d[NP];
  const T h0 = DH ? v[0] : v[0] - T(L::w(0));
  T drho = h0;
  T jx = T(0), jy = T(0), jz = T(0);
  bool ix = false, iy = false, iz = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    s[k] = DH ? v[q] + v[q + 1] : (v[q] + v[q + 1]) - T(2.0 * L::w(q));
    d[k] = v[q] - v[q + 1];
    drho += s[k];
    acc_signed(jx, ix, L::cx(q), d[k]);
    acc_signed(jy, iy, L::cy(q), d[k]);
    acc_signed(jz, iz, L::cz(q), d[k]);
  }
  T F[3] = {T(0), T(0), T(0)};
  const bool force = p.has_force != 0;
  if (force) {
    F[0] = T(p.F[0]); F[1] = T(p.F[1]); F[2] = T(p.F[2]);
    jx += T(0.5) * F[0]; jy += T(0.5) * F[1]; jz += T(0.5) * F[2];
  }
  const T rho0 = p.incompressible ? T(1) : T(1) + drho;
  const T inv = T(1) / rho0;
  const T u[3] = {jx * inv, jy * inv, L::D == 3 ? jz * inv : T(0)};
  const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T base = drho - T(1.5) * rho0 * usq;
  const T k45 = T(4.5) * rho0;
  constexpr bool SRT = OP == OP_SRT || OP == OP_SRT_LES;
  constexpr bool LES = OP == OP_SRT_LES || OP == OP_TRT_LES;
  T oe = rate<T>(p, 0);
  T oo = SRT ? oe : rate<T>(p, 1);
  if constexpr (LES) {
    // Smagorinsky (Sec. III-C): Pi^neq from the pair sums of g = h - h^eq
    // (even in c, so only s - 2 h^eq+ enters); tau from the quadratic
    // 2 tau^2 - 2 tau_0 tau - 9 C_S^2 sqrt(2 Pi:Pi) / rho = 0
    T pxx = T(0), pyy = T(0), pzz = T(0), pxy = T(0), pxz = T(0), pyz = T(0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int q = 2 * k + 1;
      const T cu = cdot<L, T>(q, u);
      const T g = s[k] - T(2.0 * L::w(q)) * fma(k45, cu * cu, base);
      const int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
      if (cx) pxx += g;
      if (cy) pyy += g;
      if (cz) pzz += g;
      if (cx && cy) pxy += cx * cy > 0 ? g : -g;
      if (cx && cz) pxz += cx * cz > 0 ? g : -g;
      if (cy && cz) pyz += cy * cz > 0 ? g : -g;
    }
    const T P = sqrt(T(2) * (pxx * pxx + pyy * pyy + pzz * pzz + T(2) * (pxy * pxy + pxz * pxz + pyz * pyz)));
    const T tau0 = T(p.smag_tau0);
    const T tau = T(0.5) * (tau0 + sqrt(tau0 * tau0 + T(p.smag_18cs2) * P / (T(1) + drho)));
    oe = T(1) / tau;
    if (SRT) oo = oe;
    else if (p.smag_magic) oo = T(1) / (T(p.smag_lambda) / (tau - T(0.5)) + T(0.5));
  }
  const T c1 = T(0.5) - T(0.5) * oe, c2 = T(0.5) - T(0.5) * oo;
  const T m3o = T(3) * rho0 * oo, m3 = T(3) * rho0;
  const T ge = T(1) - T(0.5) * oe, go = T(1) - T(0.5) * oo;
  const T uF3 = T(3) * (u[0] * F[0] + u[1] * F[1] + u[2] * F[2]);
  {
    T r0 = h0 - oe * (h0 - T(L::w(0)) * base);
    if (force) r0 -= ge * T(L::w(0)) * uF3;
    v[0] = DH ? r0 : T(L::w(0)) + r0;
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    const T w = T(L::w(q));
    const T cu = cdot<L, T>(q, u);
    T A = fma(c1, s[k], (oe * w) * fma(k45, cu * cu, base));
    if (force) {
      // Odd part as d/2 + X with X = -omega_o (d/2 - h^eq-) + (1 - omega_o/2)
      // G-: the Guo term G- = 3 w_q c_q.F is the same constant in every
      // cell, and added to a value on the coarse FP32 grid of the
      // populations it would be rounded by the same amount in every cell of
      // a binade, biasing the injected momentum (1e-4 of F at F = 1e-6,
      // |h| ~ 1e-3).  X is a small, varying non-equilibrium term, so the
      // constant is rounded on a fine grid and the final rounding of
      // d/2 + X is unbiased.
      const T cF = cdot<L, T>(q, F);
      A += ge * w * (T(9) * cu * cF - uF3);
      const T X = fma(go * w * T(3), cF, -oo * fma(T(0.5), d[k], -(m3 * w) * cu));
      const T B = fma(T(0.5), d[k], X);
      v[q] = DH ? A + B : w + (A + B);
      v[q + 1] = DH ? A - B : w + (A - B);
    } else {
      const T B = fma(c2, d[k], (m3o * w) * cu);
      v[q] = DH ? A + B : w + (A + B);
      v[q + 1] = DH ? A - B : w + (A - B);
    }
  }
}

// ---------------------------------------------------------------------- KBC
// Entropic KBC (Sec. III-C, Eq. entropic_linear_update with a fixed bulk
// rate): f - f^eq = Ds + Db + Dh with Ds the traceless and Db the trace part
// of the second-order (Hermite) projection and Dh everything of order >= 3.
// On D2Q9, D3Q19 and D3Q27 (sum w c_a^4 = 3 cs^4, sum w c_a^2 c_b^2 = cs^4)
// the w-orthogonal projections are closed forms of Pi^neq:
//   Ds_q = 4.5 w_q c_q . dev(Pi^neq) . c_q,
//   Db_q = (4.5 / D) w_q (|c_q|^2 - D/3) tr(Pi^neq).
// Both are even in c, so they live on the pair sums.  With
// X = (1 - omega_s) Ds + (1 - omega_b) Db the post-collision state is
//   f' = f^eq + X + (1 - omega_h) Dh,  1 - omega_h = -<X, Dh>_E / <Dh, Dh>_E
// (the linearised entropy condition, Eq. entropic_direct_omega_eq), with
// <a, b>_E = sum a b / f^eq.  Works on h = f - w; no body force.  Passes over
// the pairs: moments; Pi^neq; projections, the two scalar products and
// h^eq + X; then the (1 - omega_h) Dh term.
//
// 1/x for the entropic weights: the PTX approximate reciprocal in FP32
// (rcp.approx.ftz.f32; the arguments are values of f^eq, far from the
// subnormal range), an IEEE division in FP64
template <class T> __device__ __forceinline__ T kbc_rcp(T x);
template <> __device__ __forceinline__ float kbc_rcp<float>(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <> __device__ __forceinline__ double kbc_rcp<double>(double x) { return 1.0 / x; }

template <class L, class T>
__device__ __forceinline__ T kbc_quad(int q, const T (&pd)[6]) {
  // c . P . c for the symmetric P stored as (xx, yy, zz, xy, xz, yz)
  const int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
  T r = T(0);
  if (cx) r += pd[0];
  if (cy) r += pd[1];
  if (cz) r += pd[2];
  if (cx && cy) r += cx * cy > 0 ? T(2) * pd[3] : T(-2) * pd[3];
  if (cx && cz) r += cx * cz > 0 ? T(2) * pd[4] : T(-2) * pd[4];
  if (cy && cz) r += cy * cz > 0 ? T(2) * pd[5] : T(-2) * pd[5];
  return r;
}

template <class L, class T>
__device__ __forceinline__ void collide_kbc(T (&v)[L::Q], const CollideParams& p) {
  constexpr int NP = (L::Q - 1) / 2;
  constexpr int D = L::D;
  T e[NP], o[NP];
  const T h0 = v[0];
  T drho = h0;
  T jx = T(0), jy = T(0), jz = T(0);
  bool ix = false, iy = false, iz = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    e[k] = v[q] + v[q + 1];
    o[k] = v[q] - v[q + 1];
    drho += e[k];
    acc_signed(jx, ix, L::cx(q), o[k]);
    acc_signed(jy, iy, L::cy(q), o[k]);
    acc_signed(jz, iz, L::cz(q), o[k]);
  }
  const T rho0 = p.incompressible ? T(1) : T(1) + drho;
  const T inv = T(1) / rho0;
  const T u[3] = {jx * inv, jy * inv, D == 3 ? jz * inv : T(0)};
  const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T base = drho - T(1.5) * rho0 * usq;
  const T k45 = T(4.5) * rho0;
  const T m3 = T(3) * rho0;
  // pair sums and differences of f - f^eq (halved): e_k, o_k; Pi^neq from e
  T pn[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    const T w = T(L::w(q));
    const T cu = cdot<L, T>(q, u);
    const T g = e[k] - T(2) * w * fma(k45, cu * cu, base);
    const int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
    if (cx) pn[0] += g;
    if (cy) pn[1] += g;
    if (cz) pn[2] += g;
    if (cx && cy) pn[3] += cx * cy > 0 ? g : -g;
    if (cx && cz) pn[4] += cx * cz > 0 ? g : -g;
    if (cy && cz) pn[5] += cy * cz > 0 ? g : -g;
    e[k] = T(0.5) * g;
    o[k] = T(0.5) * o[k] - m3 * w * cu;
  }
  const T tr = pn[0] + pn[1] + pn[2];
  const T mean = tr * T(1.0 / D);
  pn[0] -= mean; pn[1] -= mean; pn[2] -= mean;
  if (D == 2) pn[2] = T(0);
  const T cs1 = T(1) - rate<T>(p, 0), cb1 = T(1) - rate<T>(p, 1);
  const T kb = T(4.5 / D) * tr;
  // X_q / w_q = (1 - omega_s) 4.5 c.dev.c + (1 - omega_b) (4.5/D)(|c|^2 - D/3) tr
  // e_k <- Dh even part = e_k - (Ds + Db)_q; rest: Ds_0 = 0, Db_0 = -1.5 w_0 tr
  const T w0 = T(L::w(0));
  const T X0 = cb1 * (T(-1.5) * w0 * tr);
  const T dh0 = (h0 - w0 * base) + T(1.5) * w0 * tr;
  const T feq0 = w0 * (T(1) + base);
  const T i0 = kbc_rcp(feq0);
  T num = X0 * dh0 * i0;
  T den = dh0 * dh0 * i0;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    const T w = T(L::w(q));
    const T cu = cdot<L, T>(q, u);
    const int c2 = L::cx(q) * L::cx(q) + L::cy(q) * L::cy(q) + L::cz(q) * L::cz(q);
    const T ds = T(4.5) * w * kbc_quad<L, T>(q, pn);
    const T db = w * kb * T(c2 - D / 3.0);
    const T X = cs1 * ds + cb1 * db;
    e[k] -= ds + db;
    const T a = fma(k45, cu * cu, base);
    const T E = fma(w, a, w);  // f^eq_q = E + O, f^eq_qbar = E - O
    const T O = (m3 * w) * cu;
    const T hp = e[k] + o[k], hm = e[k] - o[k];  // Dh_q, Dh_qbar
    const T tp = hp * kbc_rcp(E + O), tm = hm * kbc_rcp(E - O);
    num = fma(X, tp + tm, num);
    den = fma(tp, hp, fma(tm, hm, den));
    // h^eq + X now, (1 - omega_h) Dh once omega_h is known
    const T A0 = fma(w, a, X);
    v[q] = A0 + O;
    v[q + 1] = A0 - O;
    e[k] = hp;
    o[k] = hm;
  }
  const T mh = den > T(1e-30) ? -num / den : T(0);  // 1 - omega_h
  v[0] = fma(mh, dh0, w0 * base + X0);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    v[q] = fma(mh, e[k], v[q]);
    v[q + 1] = fma(mh, o[k], v[q + 1]);
  }
}

// -------------------------------------------- MRT with one higher-order rate
// MRT (Eq. mrt) with the w-orthogonal basis when every moment of order >= 3
// relaxes with one rate omega_h: then M^-1 S M = omega_s P_s + omega_b P_b +
// omega_h P_h with w-orthogonal projectors onto the shear moments, the bulk
// moment and everything of order >= 3.  With y = h - h^eq + G/2 (mass and
// momentum of y vanish: h^eq carries j + F/2, G carries F) the Guo-forced
// update  h* = h - M^-1 S M y + G  becomes
//   h* = h + G - omega_h y - (omega_s - omega_h) Ys - (omega_b - omega_h) Yb,
// Ys_q = 4.5 w_q c_q.dev(Pi_y).c_q, Yb_q = (4.5 / D) w_q (|c_q|^2 - D/3) tr Pi_y,
// Pi_y = sum c c y (the closed forms of the KBC operator above).  The result
// equals the general pair-form MRT up to rounding, at about the cost of TRT.
template <class L, class T>
__device__ __forceinline__ void collide_mrt3(T (&h)[L::Q], const CollideParams& p) {
  constexpr int NP = (L::Q - 1) / 2;
  constexpr int D = L::D;
  T s[NP], dd[NP];
  T drho = h[0], jx = T(0), jy = T(0), jz = T(0);
  bool ix = false, iy = false, iz = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    s[k] = h[q] + h[q + 1];
    dd[k] = h[q] - h[q + 1];
    drho += s[k];
    acc_signed(jx, ix, L::cx(q), dd[k]);
    acc_signed(jy, iy, L::cy(q), dd[k]);
    acc_signed(jz, iz, L::cz(q), dd[k]);
  }
  T F[3] = {T(0), T(0), T(0)};
  const bool force = p.has_force != 0;
  if (force) {
    F[0] = T(p.F[0]); F[1] = T(p.F[1]); F[2] = T(p.F[2]);
    jx += T(0.5) * F[0]; jy += T(0.5) * F[1]; jz += T(0.5) * F[2];
  }
  const T rho0 = p.incompressible ? T(1) : T(1) + drho;
  const T inv = T(1) / rho0;
  const T u[3] = {jx * inv, jy * inv, D == 3 ? jz * inv : T(0)};
  const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T base = drho - T(1.5) * rho0 * usq;
  const T k45 = T(4.5) * rho0, k3 = T(3) * rho0;
  const T uF3 = T(3) * (u[0] * F[0] + u[1] * F[1] + u[2] * F[2]);
  const T oh = rate<T>(p, 2);
  const T cs = rate<T>(p, 0) - oh, cb = rate<T>(p, 1) - oh;
  // pair sums of y (ys, kept in s) and Pi_y; odd parts need no projection
  T pn[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    const T w = T(L::w(q));
    const T cu = cdot<L, T>(q, u);
    T Gs = T(0);
    if (force) Gs = w * (T(9) * cu * cdot<L, T>(q, F) - uF3);
    const T ys = s[k] - T(2) * w * fma(k45, cu * cu, base) + Gs;
    const int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
    if (cx) pn[0] += ys;
    if (cy) pn[1] += ys;
    if (cz) pn[2] += ys;
    if (cx && cy) pn[3] += cx * cy > 0 ? ys : -ys;
    if (cx && cz) pn[4] += cx * cz > 0 ? ys : -ys;
    if (cy && cz) pn[5] += cy * cz > 0 ? ys : -ys;
    s[k] = ys;
  }
  const T tr = pn[0] + pn[1] + pn[2];
  const T mean = tr * T(1.0 / D);
  pn[0] -= mean; pn[1] -= mean; pn[2] -= mean;
  if (D == 2) pn[2] = T(0);
  const T kb = T(4.5 / D) * tr;
  {
    const T w0 = T(L::w(0));
    const T G0 = force ? -w0 * uF3 : T(0);
    const T y0 = h[0] - w0 * base + T(0.5) * G0;
    h[0] = h[0] + G0 - oh * y0 + cb * (T(1.5) * w0 * tr);
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    const T w = T(L::w(q));
    const T cu = cdot<L, T>(q, u);
    T Gs = T(0), Gd = T(0);
    if (force) {
      const T cF = cdot<L, T>(q, F);
      Gs = w * (T(9) * cu * cF - uF3);
      Gd = w * T(3) * cF;
    }
    const int c2 = L::cx(q) * L::cx(q) + L::cy(q) * L::cy(q) + L::cz(q) * L::cz(q);
    const T proj = cs * (T(4.5) * w * kbc_quad<L, T>(q, pn)) + cb * (w * kb * T(c2 - D / 3.0));
    // even part: s/2 + G+ - omega_h ys/2 - projections; odd part: d/2 + G- - omega_h yd/2
    const T hs = T(0.5) * (h[q] + h[q + 1]);
    const T hd = T(0.5) * (h[q] - h[q + 1]);
    if (force) {
      // the constant G- = 3 w c.F joins the small, varying relaxation terms
      // before the coarse populations are added (unbiased rounding, see
      // collide_pairs); yd is small, so its own Gd is rounded finely
      const T yd = dd[k] - T(2) * w * k3 * cu + Gd;
      const T X = Gs - T(0.5) * oh * s[k] - proj;
      const T B = hd - T(0.5) * oh * yd;
      h[q] = (hs + (X + Gd)) + B;
      h[q + 1] = (hs + (X - Gd)) - B;
    } else {
      const T yd = dd[k] - T(2) * w * k3 * cu;
      const T A = hs - T(0.5) * oh * s[k] - proj;
      const T B = hd - T(0.5) * oh * yd;
      h[q] = A + B;
      h[q + 1] = A - B;
    }
  }
}

// ---------------------------------------------------------------------- MRT
// compile-time entries of the basis table
template <class L, int K, int Qi>
constexpr int mrt_m = mrt::Table<L>::B.M[K][Qi];
template <class L, int K>
constexpr int mrt_group = mrt::Table<L>::B.group[K];

template <class L, class T, int K, int Qi>
__device__ __forceinline__ T mrt_acc(T acc, T g) {
  constexpr int c = mrt_m<L, K, Qi>;
  if constexpr (c == 0) return acc;
  else if constexpr (c == 1) return acc + g;
  else if constexpr (c == -1) return acc - g;
  else return fma(T(c), g, acc);
}

template <class L, class T, int K, int... Qs>
__device__ __forceinline__ T mrt_row(const T (&g)[L::Q], std::integer_sequence<int, Qs...>) {
  T acc = T(0);
  ((acc = mrt_acc<L, T, K, Qs>(acc, g[Qs])), ...);
  return acc;
}

template <class L, class T, int K, int Qi>
__device__ __forceinline__ T mrt_acc_nc(T acc, T d) {
  if constexpr (mrt_group<L, K> < 0) return acc;  // conserved: delta is zero
  else return mrt_acc<L, T, K, Qi>(acc, d);
}

template <class L, class T, int Qi, int... Ks>
__device__ __forceinline__ T mrt_col(const T (&d)[L::Q], std::integer_sequence<int, Ks...>) {
  T acc = T(0);
  ((acc = mrt_acc_nc<L, T, Ks, Qi>(acc, d[Ks])), ...);
  return acc;
}

template <class L, class T, int K>
__device__ __forceinline__ T mrt_delta(const T (&g)[L::Q], const CollideParams& p) {
  // conserved moments (group -1) have rate 0
  if constexpr (mrt_group<L, K> < 0) return T(0);
  else return mrt_factor<T>(p, K) * mrt_row<L, T, K>(g, std::make_integer_sequence<int, L::Q>{});
}

template <class L, class T, int... Ks>
__device__ __forceinline__ void mrt_forward(const T (&g)[L::Q], T (&d)[L::Q], const CollideParams& p,
                                            std::integer_sequence<int, Ks...>) {
  ((d[Ks] = mrt_delta<L, T, Ks>(g, p)), ...);
}

template <class L, class T, int... Qs>
__device__ __forceinline__ void mrt_backward(T (&h)[L::Q], const T (&d)[L::Q], const T (&G)[L::Q],
                                             std::integer_sequence<int, Qs...>) {
  ((h[Qs] = h[Qs] + G[Qs] - T(L::w(Qs)) * mrt_col<L, T, Qs>(d, std::make_integer_sequence<int, L::Q>{})), ...);
}

// nu_q = sum_k M_kq d_k over the non-conserved moments (M^T d, no weights)
template <class L, class T, int... Qs>
__device__ __forceinline__ void mrt_transpose_back(const T (&d)[L::Q], T (&nu)[L::Q],
                                                   std::integer_sequence<int, Qs...>) {
  ((nu[Qs] = mrt_col<L, T, Qs>(d, std::make_integer_sequence<int, L::Q>{})), ...);
}

// Pair form of Eq. mrt.  Every row of the w-orthogonal basis is an even or an
// odd polynomial (Gram-Schmidt never mixes parities, checked at compile time
// below), so for a pair (q, qbar) the even rows see only g_q + g_qbar and the
// odd rows only g_q - g_qbar; the back transform gives E + O for q and E - O
// for qbar.  This halves both transforms.
template <class L, int K>
constexpr int mrt_odd = mrt::Table<L>::B.order[K] % 2;

template <class L>
constexpr bool mrt_parity_ok() {
  for (int k = 0; k < L::Q; ++k) {
    const int sgn = mrt::Table<L>::B.order[k] % 2 ? -1 : 1;
    for (int q = 1; q < L::Q; q += 2)
      if (mrt::Table<L>::B.M[k][q] != sgn * mrt::Table<L>::B.M[k][q + 1]) return false;
    if (sgn < 0 && mrt::Table<L>::B.M[k][0] != 0) return false;
  }
  return true;
}

// m_K for one row from the rest value g0 and the pair sums / differences
template <class L, class T, int K, int... Ps>
__device__ __forceinline__ T mrt_row_pairs(T g0, const T (&gs)[(L::Q - 1) / 2], const T (&gd)[(L::Q - 1) / 2],
                                           std::integer_sequence<int, Ps...>) {
  T acc = mrt_odd<L, K> ? T(0) : mrt_acc<L, T, K, 0>(T(0), g0);
  if constexpr (mrt_odd<L, K>) ((acc = mrt_acc<L, T, K, 2 * Ps + 1>(acc, gd[Ps])), ...);
  else ((acc = mrt_acc<L, T, K, 2 * Ps + 1>(acc, gs[Ps])), ...);
  return acc;
}

template <class L, class T, int K>
__device__ __forceinline__ T mrt_delta_pairs(T g0, const T (&gs)[(L::Q - 1) / 2], const T (&gd)[(L::Q - 1) / 2],
                                             const CollideParams& p) {
  if constexpr (mrt_group<L, K> < 0) return T(0);
  else return mrt_factor<T>(p, K) * mrt_row_pairs<L, T, K>(g0, gs, gd, std::make_integer_sequence<int, (L::Q - 1) / 2>{});
}

// sum over the non-conserved rows of one parity of M_K,Qi * d_K
template <class L, class T, int ODD, int Qi, int K>
__device__ __forceinline__ T mrt_acc_par(T acc, T d) {
  if constexpr (mrt_group<L, K> < 0 || mrt_odd<L, K> != ODD) return acc;
  else return mrt_acc<L, T, K, Qi>(acc, d);
}

template <class L, class T, int ODD, int Qi, int... Ks>
__device__ __forceinline__ T mrt_col_par(const T (&d)[L::Q], std::integer_sequence<int, Ks...>) {
  T acc = T(0);
  ((acc = mrt_acc_par<L, T, ODD, Qi, Ks>(acc, d[Ks])), ...);
  return acc;
}

template <class L, class T, int... Ks>
__device__ __forceinline__ void mrt_forward_pairs(T g0, const T (&gs)[(L::Q - 1) / 2], const T (&gd)[(L::Q - 1) / 2],
                                                  T (&d)[L::Q], const CollideParams& p,
                                                  std::integer_sequence<int, Ks...>) {
  ((d[Ks] = mrt_delta_pairs<L, T, Ks>(g0, gs, gd, p)), ...);
}

// With a force, the Guo terms join the (small) relaxation term before the
// populations are added, so that the constant G- = 3 w c.F is not rounded on
// the coarse grid of h (see collide_pairs).
template <class L, class T, int... Ps>
__device__ __forceinline__ void mrt_backward_pairs(T (&h)[L::Q], const T (&d)[L::Q], const T (&Gs)[(L::Q - 1) / 2],
                                                   const T (&Gd)[(L::Q - 1) / 2], bool force,
                                                   std::integer_sequence<int, Ps...>) {
  constexpr auto ks = std::make_integer_sequence<int, L::Q>{};
  (([&] {
     constexpr int q = 2 * Ps + 1;
     const T E = mrt_col_par<L, T, 0, q>(d, ks);
     const T O = mrt_col_par<L, T, 1, q>(d, ks);
     const T w = T(L::w(q));
     if (force) {
       h[q] = h[q] + ((Gs[Ps] + Gd[Ps]) - w * (E + O));
       h[q + 1] = h[q + 1] + ((Gs[Ps] - Gd[Ps]) - w * (E - O));
     } else {
       h[q] = h[q] - w * (E + O);
       h[q + 1] = h[q + 1] - w * (E - O);
     }
   }()),
   ...);
}

template <class L, class T>
__device__ __forceinline__ void collide_mrt(T (&h)[L::Q], const CollideParams& p) {
  static_assert(mrt_parity_ok<L>(), "basis rows must be even or odd polynomials");
  constexpr int NP = (L::Q - 1) / 2;
  T s[NP], dd[NP];
  T drho = h[0], jx = T(0), jy = T(0), jz = T(0);
  bool ix = false, iy = false, iz = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    s[k] = h[q] + h[q + 1];
    dd[k] = h[q] - h[q + 1];
    drho += s[k];
    acc_signed(jx, ix, L::cx(q), dd[k]);
    acc_signed(jy, iy, L::cy(q), dd[k]);
    acc_signed(jz, iz, L::cz(q), dd[k]);
  }
  T F[3] = {T(0), T(0), T(0)};
  const bool force = p.has_force != 0;
  if (force) {
    F[0] = T(p.F[0]); F[1] = T(p.F[1]); F[2] = T(p.F[2]);
    jx += T(0.5) * F[0]; jy += T(0.5) * F[1]; jz += T(0.5) * F[2];
  }
  const T rho0 = p.incompressible ? T(1) : T(1) + drho;
  const T inv = T(1) / rho0;
  const T u[3] = {jx * inv, jy * inv, L::D == 3 ? jz * inv : T(0)};
  const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T base = drho - T(1.5) * rho0 * usq;
  const T k45 = T(4.5) * rho0, k3 = T(3) * rho0;
  const T uF3 = T(3) * (u[0] * F[0] + u[1] * F[1] + u[2] * F[2]);
  // g = h - h^eq + G/2 as rest value, pair sums and pair differences;
  // G+ (even part) and G- (odd part) of the Guo source per pair
  T G0 = T(0), Gs[NP], Gd[NP], gs[NP], gd[NP];
  if (force) G0 = -T(L::w(0)) * uF3;
  const T g0 = h[0] - T(L::w(0)) * base + T(0.5) * G0;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int q = 2 * k + 1;
    const T w = T(L::w(q));
    const T cu = cdot<L, T>(q, u);
    Gs[k] = T(0);
    Gd[k] = T(0);
    if (force) {
      const T cF = cdot<L, T>(q, F);
      Gs[k] = w * (T(9) * cu * cF - uF3);
      Gd[k] = w * T(3) * cF;
    }
    gs[k] = s[k] - T(2) * w * fma(k45, cu * cu, base) + Gs[k];
    gd[k] = dd[k] - T(2) * w * k3 * cu + Gd[k];
  }
  T d[L::Q];
  mrt_forward_pairs<L, T>(g0, gs, gd, d, p, std::make_integer_sequence<int, L::Q>{});
  h[0] = h[0] + G0 - T(L::w(0)) * mrt_col_par<L, T, 0, 0>(d, std::make_integer_sequence<int, L::Q>{});
  mrt_backward_pairs<L, T>(h, d, Gs, Gd, force, std::make_integer_sequence<int, NP>{});
}

}  // namespace lbm
