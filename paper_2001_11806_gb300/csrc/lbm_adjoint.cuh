// Discrete adjoint of the time step (the paper has no adjoint; this is the
// reverse-mode derivative of the forward sweep of lbm_kernels.cuh).
//
// Forward, two-array pull convention: P_t = C(S(P_{t-1})) with S the pull
// streaming (a link table plus UBB constants) and C the per-cell collision.
// Reverse: lambda_{t-1} = S^T [ C'(f_t)^T lambda_t ],  f_t = S(P_{t-1}).
//
// Collision Jacobian.  Every SRT/TRT/MRT collision with Guo forcing reads
//   h* = (I - R) h + Phi(rho, J),   Phi = R h^eq(rho, J) + (I - R/2) G(J, F),
// with h = f - w, rho = 1 + sum h, J = sum c h + F/2 = rho_0 u, and R the
// relaxation operator (SRT omega I; TRT omega_e on even, omega_o on odd pair
// parts; MRT W M^T D^-1 S M).  Hence
//   C'^T lambda = lambda - nu + a 1 + C b,   nu = R^T lambda,
//   a = d psi / d rho,  b = grad_J psi,   psi = nu . h^eq + kappa . G,
//   kappa = lambda - nu / 2,
// and psi needs only weighted moments of nu and kappa: with
//   h^eq_q = w_q [(rho - 1) + 3 c.J + (9/2 (c.J)^2 - 3/2 J.J) / rho_0],
//   G_q    = w_q [3 c.F - 3 J.F / rho_0 + 9 (c.J)(c.F) / rho_0],
//   n0 = sum w nu, n1 = sum w nu c, N2 = sum w nu c c^T (k0, k1, K2 for kappa):
//   psi = n0 (rho - 1) + 3 n1.J + (9/2 J.N2 J - 3/2 n0 J.J) / rho_0
//         + 3 k1.F + (9 J.K2 F - 3 k0 J.F) / rho_0.
// rho_0 = rho (compressible) contributes -X / rho^2 to a; the body-force
// gradient of one cell is dpsi/dF = b / 2 + 3 k1 + (9 K2 J - 3 k0 J) / rho_0.
//
// Streaming transpose.  f_q(y) = P_q(y - c_q) on a fluid link, and
// f_q(y) = P_qbar(y) (+ UBB constant) on a no-slip or inlet link, so the
// adjoint of P_q(x) receives exactly one contribution: from y = x + c_q if that
// cell is fluid, else from y = x itself through direction qbar.  The kernel
// therefore scatters mu_q(y) to lambda[q][y - c_q] or lambda[qbar][y] with
// plain stores.  Outlet links are non-linear in all of P(y) and are not
// differentiated (the API refuses contexts that have them).
#pragma once
#include "lbm_kernels.cuh"

namespace lbm {

// symmetric 3x3 as xx, yy, zz, xy, xz, yz
template <class T>
struct Sym3 {
  T xx = T(0), yy = T(0), zz = T(0), xy = T(0), xz = T(0), yz = T(0);
};

template <class L, class T>
__device__ __forceinline__ void wmoments(int q, T v, T& m0, T (&m1)[3], Sym3<T>& m2) {
  const T wv = T(L::w(q)) * v;
  const int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
  m0 += wv;
  if (cx) m1[0] += cx > 0 ? wv : -wv;
  if (cy) m1[1] += cy > 0 ? wv : -wv;
  if (cz) m1[2] += cz > 0 ? wv : -wv;
  if (cx) m2.xx += wv;
  if (cy) m2.yy += wv;
  if (cz) m2.zz += wv;
  if (cx && cy) m2.xy += (cx * cy > 0) ? wv : -wv;
  if (cx && cz) m2.xz += (cx * cz > 0) ? wv : -wv;
  if (cy && cz) m2.yz += (cy * cz > 0) ? wv : -wv;
}

template <class T>
__device__ __forceinline__ void sym_mul(const Sym3<T>& S, const T (&v)[3], T (&o)[3]) {
  o[0] = S.xx * v[0] + S.xy * v[1] + S.xz * v[2];
  o[1] = S.xy * v[0] + S.yy * v[1] + S.yz * v[2];
  o[2] = S.xz * v[0] + S.yz * v[1] + S.zz * v[2];
}

// nu = R^T lambda
template <class L, class T, int OP>
__device__ __forceinline__ void relax_transpose(const T (&lam)[L::Q], T (&nu)[L::Q], const CollideParams& p) {
  if constexpr (OP == OP_MRT) {
    T x[L::Q], dm[L::Q];
#pragma unroll
    for (int q = 0; q < L::Q; ++q) x[q] = T(L::w(q)) * lam[q];
    mrt_forward<L, T>(x, dm, p, std::make_integer_sequence<int, L::Q>{});
    mrt_transpose_back<L, T>(dm, nu, std::make_integer_sequence<int, L::Q>{});
  } else {
    const T oe = rate<T>(p, 0);
    const T oo = OP == OP_SRT ? oe : rate<T>(p, 1);
    nu[0] = oe * lam[0];
#pragma unroll
    for (int q = 1; q < L::Q; q += 2) {
      const T lp = T(0.5) * (lam[q] + lam[q + 1]);
      const T lm = T(0.5) * (lam[q] - lam[q + 1]);
      nu[q] = oe * lp + oo * lm;
      nu[q + 1] = oe * lp - oo * lm;
    }
  }
}

// nu_q = (R^T lambda)_q for SRT/TRT, from the pair (lambda_q, lambda_qbar);
// recomputed where needed instead of held in registers
template <class L, class T, int OP>
__device__ __forceinline__ T nu_pair(const T (&lam)[L::Q], int q, const CollideParams& p) {
  const T oe = rate<T>(p, 0);
  const T oo = OP == OP_SRT ? oe : rate<T>(p, 1);
  if (q == 0) return oe * lam[0];
  const int qb = opp(q);
  const T lp = T(0.5) * (lam[q] + lam[qb]);
  const T lm = T(0.5) * (lam[q] - lam[qb]);
  return oe * lp + oo * lm;
}

// The scalar a, vector b and body-force gradient of
//   mu = C'(h)^T lambda = lambda - nu + a 1 + C b
// for the cell whose streamed populations have moments drho = sum h and
// j = sum c h (before the Guo half force); nu is returned for MRT only (SRT
// and TRT recompute it with nu_pair).
template <class L, class T, int OP>
__device__ __forceinline__ void collide_vjp(T drho, const T (&jh)[3], const T (&lam)[L::Q], const CollideParams& p,
                                            T (&nu)[L::Q], T& a_out, T (&b)[3], T (&gF)[3]) {
  T J[3] = {jh[0], jh[1], jh[2]};
  const bool force = p.has_force != 0;
  T F[3] = {T(0), T(0), T(0)};
  if (force) {
    F[0] = T(p.F[0]); F[1] = T(p.F[1]); F[2] = T(p.F[2]);
    J[0] += T(0.5) * F[0]; J[1] += T(0.5) * F[1]; J[2] += T(0.5) * F[2];
  }
  const bool comp = p.incompressible == 0;
  const T rho = T(1) + drho;
  const T inv0 = comp ? T(1) / rho : T(1);
  T n0 = T(0), n1[3] = {T(0), T(0), T(0)}, k0 = T(0), k1[3] = {T(0), T(0), T(0)};
  Sym3<T> N2, K2;
  if constexpr (OP == OP_MRT) {
    relax_transpose<L, T, OP>(lam, nu, p);
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      wmoments<L, T>(q, nu[q], n0, n1, N2);
      if (force) wmoments<L, T>(q, lam[q] - T(0.5) * nu[q], k0, k1, K2);
    }
  } else {
    // SRT/TRT: nu = R^T lambda scales the even pair parts by omega_e and the
    // odd ones by omega_o, and the weights are even in c, so the weighted
    // moments of nu (and of kappa = lambda - nu/2) are those of lambda
    // scaled: orders 0 and 2 by omega_e, order 1 by omega_o.  One pass over
    // lambda instead of two over nu and kappa.
    T l0 = T(0), l1[3] = {T(0), T(0), T(0)};
    Sym3<T> L2;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) wmoments<L, T>(q, lam[q], l0, l1, L2);
    const T oe = rate<T>(p, 0);
    const T oo = OP == OP_SRT ? oe : rate<T>(p, 1);
    auto scale = [](const Sym3<T>& m, T f) {
      Sym3<T> r;
      r.xx = f * m.xx; r.yy = f * m.yy; r.zz = f * m.zz; r.xy = f * m.xy; r.xz = f * m.xz; r.yz = f * m.yz;
      return r;
    };
    n0 = oe * l0;
    for (int d = 0; d < 3; ++d) n1[d] = oo * l1[d];
    N2 = scale(L2, oe);
    if (force) {
      const T he = T(1) - T(0.5) * oe, ho = T(1) - T(0.5) * oo;
      k0 = he * l0;
      for (int d = 0; d < 3; ++d) k1[d] = ho * l1[d];
      K2 = scale(L2, he);
    }
  }
  T N2J[3];
  sym_mul(N2, J, N2J);
  const T JJ = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];
  const T JN2J = J[0] * N2J[0] + J[1] * N2J[1] + J[2] * N2J[2];
  T a = n0;
  if (comp) a -= inv0 * inv0 * (T(4.5) * JN2J - T(1.5) * n0 * JJ);
  for (int d = 0; d < 3; ++d) b[d] = T(3) * n1[d] + inv0 * (T(9) * N2J[d] - T(3) * n0 * J[d]);
  gF[0] = gF[1] = gF[2] = T(0);
  if (force) {
    T K2F[3], K2J[3];
    sym_mul(K2, F, K2F);
    sym_mul(K2, J, K2J);
    const T JF = J[0] * F[0] + J[1] * F[1] + J[2] * F[2];
    const T JK2F = J[0] * K2F[0] + J[1] * K2F[1] + J[2] * K2F[2];
    if (comp) a -= inv0 * inv0 * (T(9) * JK2F - T(3) * k0 * JF);
    for (int d = 0; d < 3; ++d) b[d] += inv0 * (T(9) * K2F[d] - T(3) * k0 * F[d]);
    for (int d = 0; d < 3; ++d) gF[d] = T(0.5) * b[d] + T(3) * k1[d] + inv0 * (T(9) * K2J[d] - T(3) * k0 * J[d]);
  }
  if (L::D == 2) { b[2] = T(0); gF[2] = T(0); }
  a_out = a;
}

// Body-force gradient of the adjoint sweep: every block writes the FP64 sum
// of its cells' contributions to its own row of a scratch array (no
// atomics: one address shared by all blocks of a 2 M-cell sweep serialised
// tens of thousands of atomic adds per step), and k_force_rows_final adds the
// rows in a fixed order to the caller's accumulator.
template <class T>
__device__ __forceinline__ void block_row3(const T (&v)[3], double* rows) {
  __shared__ double sh[kBlockX / 32][3];
  double s[3] = {double(v[0]), double(v[1]), double(v[2])};
  for (int d = 0; d < 3; ++d) s[d] = warp_sum(s[d]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) sh[wid][d] = s[d];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x + 31) / 32; ++w) t += sh[w][threadIdx.x];
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    rows[b * 3 + threadIdx.x] = t;
  }
}

// accum[0..2] += sum of rows[0 .. nrows) (one block of kForceThreads)
constexpr int kForceThreads = 256;
template <class R>
__global__ void __launch_bounds__(kForceThreads) k_force_rows_final(const R* rows, long long nrows, R* accum) {
  __shared__ R sh[kForceThreads / 32][3];
  R s[3] = {0.0, 0.0, 0.0};
  for (long long r = threadIdx.x; r < nrows; r += kForceThreads)
    for (int d = 0; d < 3; ++d) s[d] += rows[r * 3 + d];
  for (int d = 0; d < 3; ++d) s[d] = warp_sum(s[d]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int d = 0; d < 3; ++d) sh[wid][d] = s[d];
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kForceThreads / 32; ++w) t += sh[w][threadIdx.x];
    accum[threadIdx.x] += t;
  }
}

template <class T>
__device__ __forceinline__ void block_add3(T (&v)[3], double* accum) {
  // warp sums, then one FP64 atomic per warp and component
  double s[3] = {double(v[0]), double(v[1]), double(v[2])};
  for (int d = 0; d < 3; ++d) s[d] = warp_sum(s[d]);
  if ((threadIdx.x & 31) == 0)
    for (int d = 0; d < 3; ++d)
      if (s[d] != 0.0) atomicAdd(&accum[d], s[d]);
}

// Pull-load of f(y) as shifted populations h (no-slip and inlet links; the
// API guarantees there are no outlet links).
template <class L, class ST, bool BND>
__device__ __forceinline__ void pull_h(const SweepArgs& a, const Nbr& nb, int cell, uint32_t mask,
                                       typename ST::T (&h)[L::Q]) {
  using S = typename ST::S;
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    const bool b = BND && ((mask >> q) & 1u);
    const int qs = b ? opp(q) : q;
    const int idx = b ? cell : nb.at(-L::cx(q), -L::cy(q), -L::cz(q));
    h[q] = ST::to_h(reinterpret_cast<const S*>(a.srcq[qs])[idx], L::w(q));
  }
}

template <class L, class T, bool BND>
__device__ __forceinline__ void inlet_fix(const SweepArgs& a, int x, int y, int z, uint32_t mask, T (&h)[L::Q]) {
  if constexpr (BND) {
    if (mask & MASK_SPECIAL) {
      for (int q = 1; q < L::Q; ++q) {
        if ((mask >> q) & 1u) {
          const int t = LBM_LINK_TYPE(a, x - L::cx(q), y - L::cy(q), z - L::cz(q));
          if (t == L_INLET) h[q] += ubb_term<L, T>(q, a.cp);
        }
      }
    }
  }
}

// Scatter mu(y) through the transposed streaming map.
template <class L, class T, bool BND>
__device__ __forceinline__ void scatter_T(const SweepArgs& a, const Nbr& nb, int cell, uint32_t mask,
                                          const T (&mu)[L::Q], T* lam_out) {
  const long long N = a.g.N;
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    const bool b = BND && ((mask >> q) & 1u);
    const int qd = b ? opp(q) : q;
    const int idx = b ? cell : nb.at(-L::cx(q), -L::cy(q), -L::cz(q));
    lam_out[qd * N + idx] = mu[q];
  }
}

// A global load the compiler may not merge with an earlier load of the same
// address (asm volatile), so the earlier value need not stay in a register.
__device__ __forceinline__ float reload(const float* p) {
  float v;
  asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double reload(const double* p) {
  double v;
  asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// The adjoint sweep.  The forward populations f(y) = S(P_prev)(y) enter only
// through rho and j, so they are summed while loaded and not kept.  Periodic
// domains use the same pre-shifted stream bases as the forward pull sweep in
// rows whose y/z neighbours do not wrap: SweepArgs::srci for P_prev and
// SweepArgs::dsti for lambda_out (base of stream q minus the offset of c_q).
template <class L, class ST, int OP, bool BND>
__global__ void __launch_bounds__(kBlockX) k_adjoint(const SweepArgs a, const typename ST::T* lam_in,
                                                     typename ST::T* lam_out, double* force_rows) {
  using T = typename ST::T;
  using S = typename ST::S;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  T gF[3] = {T(0), T(0), T(0)};
  if (x < a.g.nx) {
    const int y = blockIdx.y, z = blockIdx.z;
    const int cell = x + a.g.nx * (y + a.g.ny * z);
    const long long N = a.g.N;
    uint32_t mask = 0;
    if constexpr (BND) mask = a.mask[cell];
    if (mask & MASK_SOLID) {
      for (int q = 0; q < L::Q; ++q) lam_out[q * N + cell] = T(0);
    } else {
      bool fast = false;
      if constexpr (!BND) fast = row_inner<L>(a.g, y, z);
      const int im = cell + (x == 0 ? a.g.nx : 0);
      const int ip = cell - (x == a.g.nx - 1 ? a.g.nx : 0);
      T drho = T(0), jh[3] = {T(0), T(0), T(0)};
      if (fast) {
#pragma unroll
        for (int q = 0; q < L::Q; ++q) {
          const int idx = L::cx(q) > 0 ? im : (L::cx(q) < 0 ? ip : cell);
          const T hq = ST::to_h(reinterpret_cast<const S*>(a.srci[q])[idx], L::w(q));
          drho += hq;
          jh[0] += T(L::cx(q)) * hq; jh[1] += T(L::cy(q)) * hq; jh[2] += T(L::cz(q)) * hq;
        }
      } else {
        const Nbr nb = make_nbr(a.g, x, y, z);
#pragma unroll
        for (int q = 0; q < L::Q; ++q) {
          const bool b = BND && ((mask >> q) & 1u);
          const int qs = b ? opp(q) : q;
          const int idx = b ? cell : nb.at(-L::cx(q), -L::cy(q), -L::cz(q));
          const T hq = ST::to_h(reinterpret_cast<const S*>(a.srcq[qs])[idx], L::w(q));
          drho += hq;
          jh[0] += T(L::cx(q)) * hq; jh[1] += T(L::cy(q)) * hq; jh[2] += T(L::cz(q)) * hq;
        }
        if constexpr (BND) {
          // inlet links carry the UBB constant (no outlet links here)
          if (mask & MASK_SPECIAL) {
            for (int q = 1; q < L::Q; ++q) {
              if ((mask >> q) & 1u) {
                if (LBM_LINK_TYPE(a, x - L::cx(q), y - L::cy(q), z - L::cz(q)) == L_INLET) {
                  const T u = ubb_term<L, T>(q, a.cp);
                  drho += u;
                  jh[0] += T(L::cx(q)) * u; jh[1] += T(L::cy(q)) * u; jh[2] += T(L::cz(q)) * u;
                }
              }
            }
          }
        }
      }
      T lam[L::Q], nu[L::Q];
#pragma unroll
      for (int q = 0; q < L::Q; ++q) lam[q] = lam_in[q * N + cell];
      T av, bv[3];
      collide_vjp<L, T, OP>(drho, jh, lam, a.cp, nu, av, bv, gF);
      // scatter mu(y) through the transposed streaming map; SRT/TRT read
      // lambda again (a cache hit) instead of holding it across the moments
      if constexpr (OP != OP_MRT) {
#pragma unroll
        for (int q = 0; q < L::Q; ++q) lam[q] = reload(lam_in + q * N + cell);
      }
#pragma unroll
      for (int q = 0; q < L::Q; ++q) {
        const T nq = OP == OP_MRT ? nu[q] : nu_pair<L, T, OP>(lam, q, a.cp);
        const T mu = lam[q] - nq + av + T(L::cx(q)) * bv[0] + T(L::cy(q)) * bv[1] + T(L::cz(q)) * bv[2];
        if (fast) {
          const int idx = L::cx(q) > 0 ? im : (L::cx(q) < 0 ? ip : cell);
          reinterpret_cast<T*>(a.dsti[q])[idx] = mu;
        } else {
          const Nbr nb = make_nbr(a.g, x, y, z);
          const bool b = BND && ((mask >> q) & 1u);
          const int qd = b ? opp(q) : q;
          const int idx = b ? cell : nb.at(-L::cx(q), -L::cy(q), -L::cz(q));
          lam_out[qd * N + idx] = mu;
        }
      }
    }
  }
  if (force_rows != nullptr) block_row3(gF, force_rows);
}

// Kinetic energy in a box, L = (1/2) sum_{x in box, fluid} rho |u|^2 of the
// populations f = S(P), and the seed lambda = S^T dL/df.
template <class L, class ST, bool BND>
__global__ void __launch_bounds__(kBlockX) k_ke_seed(const SweepArgs a, int4 lo, int4 hi, double* L_out,
                                                     typename ST::T* lam_out, double* dLdF) {
  using T = typename ST::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  T gF[3] = {T(0), T(0), T(0)};
  if (x < a.g.nx) {
    const int y = blockIdx.y, z = blockIdx.z;
    const int cell = x + a.g.nx * (y + a.g.ny * z);
    const long long N = a.g.N;
    uint32_t mask = 0;
    if constexpr (BND) mask = a.mask[cell];
    if (mask & MASK_SOLID) {
      if (lam_out)
        for (int q = 0; q < L::Q; ++q) lam_out[q * N + cell] = T(0);
    } else {
      const Nbr nb = make_nbr(a.g, x, y, z);
      T h[L::Q], mu[L::Q];
      const bool in_box = x >= lo.x && x < hi.x && y >= lo.y && y < hi.y && z >= lo.z && z < hi.z;
      if (in_box) {
        pull_h<L, ST, BND>(a, nb, cell, mask, h);
        inlet_fix<L, T, BND>(a, x, y, z, mask, h);
        T drho = T(0), J[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int q = 0; q < L::Q; ++q) {
          drho += h[q];
          J[0] += T(L::cx(q)) * h[q];
          J[1] += T(L::cy(q)) * h[q];
          J[2] += T(L::cz(q)) * h[q];
        }
        if (a.cp.has_force)
          for (int d = 0; d < 3; ++d) J[d] += T(0.5 * a.cp.F[d]);
        if (L::D == 2) J[2] = T(0);
        const T rho = T(1) + drho;
        const T JJ = J[0] * J[0] + J[1] * J[1] + J[2] * J[2];
        T de_drho, de_dJ[3];
        if (a.cp.incompressible) {  // e = rho |J|^2 / 2
          e = 0.5 * double(rho) * double(JJ);
          de_drho = T(0.5) * JJ;
          for (int d = 0; d < 3; ++d) de_dJ[d] = rho * J[d];
        } else {  // e = |J|^2 / (2 rho)
          const T inv = T(1) / rho;
          e = 0.5 * double(JJ) / double(rho);
          de_drho = T(-0.5) * JJ * inv * inv;
          for (int d = 0; d < 3; ++d) de_dJ[d] = J[d] * inv;
        }
        for (int q = 0; q < L::Q; ++q)
          mu[q] = de_drho + T(L::cx(q)) * de_dJ[0] + T(L::cy(q)) * de_dJ[1] + T(L::cz(q)) * de_dJ[2];
        if (a.cp.has_force)
          for (int d = 0; d < 3; ++d) gF[d] = T(0.5) * de_dJ[d];
      } else {
        for (int q = 0; q < L::Q; ++q) mu[q] = T(0);
      }
      if (lam_out) scatter_T<L, T, BND>(a, nb, cell, mask, mu, lam_out);
    }
  }
  const double es = warp_sum(e);
  if ((threadIdx.x & 31) == 0 && es != 0.0) atomicAdd(L_out, es);
  if (dLdF != nullptr && a.cp.has_force) block_add3(gF, dLdF);
}

// g_u0 = (d f^eq(rho_0, u_0) / d u_0)^T lambda per fluid cell, FP64:
// d f^eq_q / d u = w_q rho_0 (3 c_q + 9 (c_q.u) c_q - 3 u).
template <class L, class T>
__global__ void k_eq_vjp(const SweepArgs a, const double* rho0, const double* u0, const T* lam, double* g) {
  const long long N = a.g.N;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    const uint32_t mask = a.mask ? a.mask[cell] : 0u;
    double out[3] = {0, 0, 0};
    if (!(mask & MASK_SOLID)) {
      const double r0 = a.cp.incompressible ? 1.0 : rho0[cell];
      const double u[3] = {u0[cell], u0[N + cell], L::D == 3 ? u0[2 * N + cell] : 0.0};
      double l0 = 0, l1[3] = {0, 0, 0};
      Sym3<double> L2;
      for (int q = 0; q < L::Q; ++q) wmoments<L, double>(q, double(lam[q * N + cell]), l0, l1, L2);
      double L2u[3];
      sym_mul(L2, u, L2u);
      for (int d = 0; d < 3; ++d) out[d] = r0 * (3.0 * l1[d] + 9.0 * L2u[d] - 3.0 * l0 * u[d]);
    }
    for (int d = 0; d < L::D; ++d) g[d * N + cell] = out[d];
  }
}

}  // namespace lbm
