// D3Q27 cumulant collision (Sec. III-B, Eq. cumulant_generating_function).
//
// Populations -> central moments -> cumulants -> relax -> back, the
// multi-step route of Sec. III-B with moments as intermediate quantities:
//   1. per-axis central-moment transform (z, then y, then x) of the 27
//      populations about the cell velocity u = j / rho: for each line of
//      three populations (c = -1, 0, +1) along an axis,
//        m0 = sum f, m1 = sum (c - u) f, m2 = sum (c - u)^2 f;
//   2. normalised central moments C = m / rho; cumulants of order 2 and 3
//      equal them; orders 4-6 follow from ln of the moment generating
//      function (first-order central moments vanish), e.g.
//        k220 = C220 - C200 C020 - 2 C110^2,
//        k211 = C211 - C200 C011 - 2 C110 C101,
//        k221 = C221 - C200 C021 - C020 C201 - 4 C110 C111
//               - 2 C101 C120 - 2 C011 C210,
//        k222 = C222 - (C200 C022 + C020 C202 + C002 C220)
//               - 4 (C110 C112 + C101 C121 + C011 C211)
//               - 2 (C210 C012 + C201 C021 + C120 C102) - 4 C111^2
//               + 2 C200 C020 C002 + 16 C110 C101 C011
//               + 4 (C200 C011^2 + C020 C101^2 + C002 C110^2);
//   3. relaxation: off-diagonal second-order cumulants and the two diagonal
//      differences with omega_shear toward 0, the trace with omega_bulk
//      toward 3 c_s^2 = 1, every order >= 3 with omega_higher toward 0;
//      rho and u are conserved;
//   4. post-collision central moments from the relaxed cumulants (the same
//      relations solved for C, using post-collision lower orders), then the
//      inverse per-axis transform
//        f(-1) = (m0 (u^2 - u) + m1 (2u - 1) + m2) / 2,
//        f( 0) = m0 (1 - u^2) - 2 u m1 - m2,
//        f(+1) = (m0 (u^2 + u) + m1 (2u + 1) + m2) / 2.
#pragma once
#include "lbm_collide.cuh"

namespace lbm {

__host__ __device__ constexpr int slot27(int q) {
  return 9 * (D3Q27::cx(q) + 1) + 3 * (D3Q27::cy(q) + 1) + (D3Q27::cz(q) + 1);
}

// With t = f(+1) - f(-1) and S = f(+1) + f(-1) of a line:
//   m0 = S + f(0),  m1 = t - u m0,  m2 = S - 2 u t + u^2 m0 = S - u (t + m1),
// and back: t = m1 + u m0, S = m2 + u (m1 + t), f(0) = m0 - S,
// f(+-1) = (S +- t) / 2.
template <class T>
__device__ __forceinline__ void chimera_fwd(T& a, T& b, T& c, T u) {
  const T S = c + a, t = c - a;
  const T m0 = S + b;
  const T m1 = fma(-u, m0, t);
  a = m0;
  b = m1;
  c = fma(-u, t + m1, S);
}

// the central part of chimera_fwd for a line already holding (m0, t, S)
template <class T>
__device__ __forceinline__ void chimera_shift(T& b, T& c, T m0, T u) {
  const T t = b;
  const T m1 = fma(-u, m0, t);
  b = m1;
  c = fma(-u, t + m1, c);
}

template <class T>
__device__ __forceinline__ void chimera_bwd(T& a, T& b, T& c, T u) {
  const T m0 = a, m1 = b, m2 = c;
  const T t = fma(u, m0, m1);
  const T S = fma(u, m1 + t, m2);
  const T ht = T(0.5) * t;
  a = fma(T(0.5), S, -ht);
  b = m0 - S;
  c = fma(T(0.5), S, ht);
}

#define LBM_C(a, b, c) F[9 * (a) + 3 * (b) + (c)]

// Both transforms run on deviations from the rest state (rho = 1, u = 0,
// f = w) so that every intermediate is small and FP32 keeps its relative
// precision on the small populations.  The transform is linear and the rest
// weights are a product of 1-D weights, so their central moments about u are
// known in closed form: mu_0 = 1, mu_1 = -u, mu_2 = 1/3 + u^2 per axis, and
//   C_abc = H_abc + mu_a(u_x) mu_b(u_y) mu_c(u_z),   H = transform of h.
// Second-order diagonal moments are carried as e = C/rho - 1/3, fourth-order
// diagonal ones as E = C/rho - 1/9, the sixth-order one as E = C/rho - 1/27;
// the cumulant relations above are expanded in these deviations so that the
// large rest-state constants cancel analytically.  After relaxation the
// deviations of the post-collision moments from the rest-state moments are
// transformed back, which yields h* = f* - w directly.
template <class T>
__device__ __forceinline__ void collide_cumulant(T (&h)[27], const CollideParams& p) {
  T F[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) F[slot27(q)] = h[q];
  // z lines first as raw sums (m0, t, S); rho and j follow from them: line i
  // has c_x = i / 3 - 1, c_y = i % 3 - 1
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T a = F[3 * i], b = F[3 * i + 1], c = F[3 * i + 2];
    const T S = c + a;
    F[3 * i] = S + b;
    F[3 * i + 1] = c - a;
    F[3 * i + 2] = S;
  }
  T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    drho += F[3 * i];
    jz += F[3 * i + 1];
    if (i / 3 == 2) jx += F[3 * i];
    if (i / 3 == 0) jx -= F[3 * i];
    if (i % 3 == 2) jy += F[3 * i];
    if (i % 3 == 0) jy -= F[3 * i];
  }
  const T rho = T(1) + drho;
  const T inv = T(1) / rho;
  const T ux = jx * inv, uy = jy * inv, uz = jz * inv;
  // forward transform of h: z lines (central part), y lines, x lines
#pragma unroll
  for (int i = 0; i < 9; ++i) chimera_shift(F[3 * i + 1], F[3 * i + 2], F[3 * i], uz);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) chimera_fwd(F[9 * i + k], F[9 * i + 3 + k], F[9 * i + 6 + k], uy);
#pragma unroll
  for (int j = 0; j < 9; ++j) chimera_fwd(F[j], F[9 + j], F[18 + j], ux);

  const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0), two = T(2), four = T(4);
  const T x2 = ux * ux, y2 = uy * uy, z2 = uz * uz, usq = x2 + y2 + z2;
  const T m2x = third + x2, m2y = third + y2, m2z = third + z2;
  // normalised pre-collision central moments (deviation form)
  const T a = (LBM_C(2, 0, 0) + x2 - drho * third) * inv;
  const T b = (LBM_C(0, 2, 0) + y2 - drho * third) * inv;
  const T c = (LBM_C(0, 0, 2) + z2 - drho * third) * inv;
  const T C110 = (LBM_C(1, 1, 0) + ux * uy) * inv;
  const T C101 = (LBM_C(1, 0, 1) + ux * uz) * inv;
  const T C011 = (LBM_C(0, 1, 1) + uy * uz) * inv;
  const T om = rate<T>(p, 0), omb = rate<T>(p, 1), omh = rate<T>(p, 2);
  const T rs = T(1) - om, rh = T(1) - omh;
  // Orders >= 3 enter the post-collision state only as rh * (pre-collision
  // moment or cumulant); with omega_higher = 1 (rh = 0, a uniform branch)
  // they are not formed at all.  r... = rh * k... below.
  T P210 = T(0), P201 = T(0), P120 = T(0), P021 = T(0), P102 = T(0), P012 = T(0), P111 = T(0);
  T r220 = T(0), r202 = T(0), r022 = T(0), r211 = T(0), r121 = T(0), r112 = T(0);
  T r221 = T(0), r212 = T(0), r122 = T(0), r222 = T(0);
  if (rh != T(0)) {
    const T C210 = (LBM_C(2, 1, 0) - m2x * uy) * inv, C201 = (LBM_C(2, 0, 1) - m2x * uz) * inv;
    const T C120 = (LBM_C(1, 2, 0) - m2y * ux) * inv, C021 = (LBM_C(0, 2, 1) - m2y * uz) * inv;
    const T C102 = (LBM_C(1, 0, 2) - m2z * ux) * inv, C012 = (LBM_C(0, 1, 2) - m2z * uy) * inv;
    const T C111 = (LBM_C(1, 1, 1) - ux * uy * uz) * inv;
    const T E220 = (LBM_C(2, 2, 0) + (x2 + y2) * third + x2 * y2 - drho * ninth) * inv;
    const T E202 = (LBM_C(2, 0, 2) + (x2 + z2) * third + x2 * z2 - drho * ninth) * inv;
    const T E022 = (LBM_C(0, 2, 2) + (y2 + z2) * third + y2 * z2 - drho * ninth) * inv;
    const T C211 = (LBM_C(2, 1, 1) + m2x * uy * uz) * inv;
    const T C121 = (LBM_C(1, 2, 1) + m2y * ux * uz) * inv;
    const T C112 = (LBM_C(1, 1, 2) + m2z * ux * uy) * inv;
    const T C221 = (LBM_C(2, 2, 1) - m2x * m2y * uz) * inv;
    const T C212 = (LBM_C(2, 1, 2) - m2x * m2z * uy) * inv;
    const T C122 = (LBM_C(1, 2, 2) - m2y * m2z * ux) * inv;
    const T E222 = (LBM_C(2, 2, 2) + usq * ninth + (x2 * y2 + y2 * z2 + z2 * x2) * third + x2 * y2 * z2 -
                    drho * T(1.0 / 27.0)) * inv;
    // pre-collision cumulants of order 4-6 (the relations of the header with
    // C200 = 1/3 + a, C220 = 1/9 + E220, C222 = 1/27 + E222, ...)
    const T k220 = E220 - (a + b) * third - a * b - two * C110 * C110;
    const T k202 = E202 - (a + c) * third - a * c - two * C101 * C101;
    const T k022 = E022 - (b + c) * third - b * c - two * C011 * C011;
    const T k211 = C211 - (third + a) * C011 - two * C110 * C101;
    const T k121 = C121 - (third + b) * C101 - two * C110 * C011;
    const T k112 = C112 - (third + c) * C110 - two * C101 * C011;
    const T k221 = C221 - (third + a) * C021 - (third + b) * C201 - four * C110 * C111 - two * C101 * C120 -
                   two * C011 * C210;
    const T k212 = C212 - (third + a) * C012 - (third + c) * C210 - four * C101 * C111 - two * C110 * C102 -
                   two * C011 * C201;
    const T k122 = C122 - (third + b) * C102 - (third + c) * C120 - four * C011 * C111 - two * C110 * C012 -
                   two * C101 * C021;
    const T k222 = E222 - (E220 + E202 + E022) * third + (a + b + c) * ninth - (a * E022 + b * E202 + c * E220) +
                   T(2.0 / 3.0) * (a * b + b * c + c * a) + two * a * b * c -
                   four * (C110 * C112 + C101 * C121 + C011 * C211) -
                   two * (C210 * C012 + C201 * C021 + C120 * C102) - four * C111 * C111 +
                   T(16) * C110 * C101 * C011 +
                   four * ((third + a) * C011 * C011 + (third + b) * C101 * C101 + (third + c) * C110 * C110);
    P210 = rh * C210; P201 = rh * C201; P120 = rh * C120;
    P021 = rh * C021; P102 = rh * C102; P012 = rh * C012; P111 = rh * C111;
    r220 = rh * k220; r202 = rh * k202; r022 = rh * k022;
    r211 = rh * k211; r121 = rh * k121; r112 = rh * k112;
    r221 = rh * k221; r212 = rh * k212; r122 = rh * k122; r222 = rh * k222;
  }
  // relaxation: shear (off-diagonals and diagonal differences), bulk (trace
  // toward 3 c_s^2, i.e. a + b + c toward 0), higher orders toward 0
  const T d1 = rs * (a - b), d2 = rs * (a - c), tm1 = (T(1) - omb) * (a + b + c);
  const T A = (tm1 + d1 + d2) * third, B = (tm1 - two * d1 + d2) * third, Cc = (tm1 + d1 - two * d2) * third;
  const T P110 = rs * C110, P101 = rs * C101, P011 = rs * C011;
  const T Q220 = r220 + (A + B) * third + A * B + two * P110 * P110;
  const T Q202 = r202 + (A + Cc) * third + A * Cc + two * P101 * P101;
  const T Q022 = r022 + (B + Cc) * third + B * Cc + two * P011 * P011;
  const T P211 = r211 + (third + A) * P011 + two * P110 * P101;
  const T P121 = r121 + (third + B) * P101 + two * P110 * P011;
  const T P112 = r112 + (third + Cc) * P110 + two * P101 * P011;
  const T P221 = r221 + (third + A) * P021 + (third + B) * P201 + four * P110 * P111 + two * P101 * P120 +
                 two * P011 * P210;
  const T P212 = r212 + (third + A) * P012 + (third + Cc) * P210 + four * P101 * P111 + two * P110 * P102 +
                 two * P011 * P201;
  const T P122 = r122 + (third + B) * P102 + (third + Cc) * P120 + four * P011 * P111 + two * P110 * P012 +
                 two * P101 * P021;
  const T Q222 = r222 + (Q220 + Q202 + Q022) * third - (A + B + Cc) * ninth +
                 (A * Q022 + B * Q202 + Cc * Q220) - T(2.0 / 3.0) * (A * B + B * Cc + Cc * A) - two * A * B * Cc +
                 four * (P110 * P112 + P101 * P121 + P011 * P211) +
                 two * (P210 * P012 + P201 * P021 + P120 * P102) + four * P111 * P111 -
                 T(16) * P110 * P101 * P011 -
                 four * ((third + A) * P011 * P011 + (third + B) * P101 * P101 + (third + Cc) * P110 * P110);
  // deviations of the post-collision central moments from those of the rest
  // weights (rho C* - mu mu mu), un-normalised
  LBM_C(0, 0, 0) = drho;
  LBM_C(1, 0, 0) = ux; LBM_C(0, 1, 0) = uy; LBM_C(0, 0, 1) = uz;
  LBM_C(2, 0, 0) = drho * third + rho * A - x2;
  LBM_C(0, 2, 0) = drho * third + rho * B - y2;
  LBM_C(0, 0, 2) = drho * third + rho * Cc - z2;
  LBM_C(1, 1, 0) = rho * P110 - ux * uy;
  LBM_C(1, 0, 1) = rho * P101 - ux * uz;
  LBM_C(0, 1, 1) = rho * P011 - uy * uz;
  LBM_C(2, 1, 0) = rho * P210 + m2x * uy; LBM_C(2, 0, 1) = rho * P201 + m2x * uz;
  LBM_C(1, 2, 0) = rho * P120 + m2y * ux; LBM_C(0, 2, 1) = rho * P021 + m2y * uz;
  LBM_C(1, 0, 2) = rho * P102 + m2z * ux; LBM_C(0, 1, 2) = rho * P012 + m2z * uy;
  LBM_C(1, 1, 1) = rho * P111 + ux * uy * uz;
  LBM_C(2, 2, 0) = drho * ninth + rho * Q220 - (x2 + y2) * third - x2 * y2;
  LBM_C(2, 0, 2) = drho * ninth + rho * Q202 - (x2 + z2) * third - x2 * z2;
  LBM_C(0, 2, 2) = drho * ninth + rho * Q022 - (y2 + z2) * third - y2 * z2;
  LBM_C(2, 1, 1) = rho * P211 - m2x * uy * uz;
  LBM_C(1, 2, 1) = rho * P121 - m2y * ux * uz;
  LBM_C(1, 1, 2) = rho * P112 - m2z * ux * uy;
  LBM_C(2, 2, 1) = rho * P221 + m2x * m2y * uz;
  LBM_C(2, 1, 2) = rho * P212 + m2x * m2z * uy;
  LBM_C(1, 2, 2) = rho * P122 + m2y * m2z * ux;
  LBM_C(2, 2, 2) = drho * T(1.0 / 27.0) + rho * Q222 - usq * ninth - (x2 * y2 + y2 * z2 + z2 * x2) * third -
                   x2 * y2 * z2;
  // backward transform: x lines, y lines, z lines; the result is h* = f* - w
#pragma unroll
  for (int j = 0; j < 9; ++j) chimera_bwd(F[j], F[9 + j], F[18 + j], ux);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) chimera_bwd(F[9 * i + k], F[9 * i + 3 + k], F[9 * i + 6 + k], uy);
#pragma unroll
  for (int i = 0; i < 9; ++i) chimera_bwd(F[3 * i], F[3 * i + 1], F[3 * i + 2], uz);
#pragma unroll
  for (int q = 0; q < 27; ++q) h[q] = F[slot27(q)];
}

#undef LBM_C

}  // namespace lbm
