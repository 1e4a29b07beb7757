// Stream-collide sweep kernels and their helpers.
//
// Update patterns (Sec. IV-B "Streaming and Collision"):
//   K_PULL     two arrays; cell x reads P_q(x - c_q) from src (pull), collides
//              and writes dst[q][x].
//   K_AA_EVEN  single array A; reads A[q][x], collides, writes the result of
//              direction q to A[qbar][x] (in place, inverted).
//   K_AA_ODD   reads A[qbar][x - c_q], collides, writes direction q to
//              A[q][x + c_q].  Each thread touches only its own slots, so the
//              update is race free.
// Boundaries are compiled into the sweep (Sec. IV-B "Boundary Conditions"):
// a per-cell link mask (bit q = the source x - c_q is not fluid) selects the
// boundary value B_q(P(x)) of the cell's own post-collision populations:
//   no-slip B_q = P_qbar; velocity bounce-back (UBB listing, Sec. III-C)
//   B_q = P_qbar + 2 w_q (c_q.u_w)/c_s^2; outlet B_q = f^eq_q(rho_out, u_P).
// In the AA pattern the producer of P(x) writes B_q into A[q][x] (the slot
// the missing source cell would have filled), so even and odd steps read
// boundary links like any other population.
//
// Memory layout: structure of arrays [q][N], N = nx*ny*nz, x fastest.  One
// thread per cell, consecutive threads along x, so every population stream
// is read and written by whole warps over consecutive addresses; the +-1
// x-shift of a pull only offsets a warp's window by one element.
#pragma once
#include "lbm_collide.cuh"
#include "lbm_cumulant.cuh"

namespace lbm {

enum Kind : int { K_PULL = 0, K_AA_EVEN = 1, K_AA_ODD = 2, K_ESO_EVEN = 3, K_ESO_ODD = 4 };
enum View : int { V_PULL = 0, V_AA_NATURAL = 1, V_AA_INVERTED = 2, V_ESO_EVEN = 3, V_ESO_ODD = 4 };

// Esoteric twist (Sec. IV-B, single array run as even and odd kernels).  Cell
// x owns the slots at x and at its positive neighbours: it reads f_q(x) from
// location x + max(-c_q, 0) (componentwise; slot q after an even number of
// steps, slot qbar after an odd number) and writes P_q(x) to location
// x + max(c_q, 0) (slot qbar in the even kernel, q in the odd kernel), where
// the cell x + c_q reads it in the next step.  Locations wrap on every axis;
// on a non-periodic axis the wrapped pairs are kept apart by the boundary
// rule: for a boundary link (x, qbar) the value B_qbar(P(x)) goes to the
// other slot of the same location (q in the even kernel, qbar in the odd
// one), which is the slot x reads f_qbar(x) from in the next step and which
// the link's source would have written.
__host__ __device__ constexpr int eso_rd(int c) { return c < 0 ? 1 : 0; }
// Set by k_link_mask in its types word when a fluid cell lies in the last
// layer (index n - 1) of a non-periodic axis.  The esoteric twist needs that
// layer non-fluid: its wrapped locations are shared with the first layer,
// whose boundary links would then race with the fluid cells there.
constexpr unsigned TYPES_FLUID_LAST_LAYER = 1u << 8;
// ... and when a fluid cell lies in the first layer of a non-periodic axis
// (a boundary link whose source is outside the box)
constexpr unsigned TYPES_FLUID_FIRST_LAYER = 1u << 9;
__host__ __device__ constexpr int eso_wr(int c) { return c > 0 ? 1 : 0; }

struct Geom {
  int nx, ny, nz;
  int per[3];
  long long N;
};

struct SweepArgs {
  const void* src;       // K_PULL: read array; AA: the single array
  void* dst;             // K_PULL: write array; AA: the single array
  const uint32_t* mask;  // link mask [N] or null
  const uint8_t* flags;  // flag field [N] or null
  Geom g;
  CollideParams cp;
  // start of each direction's stream in src / dst (src + q*N elements), so
  // that every population access is one 32-bit cell offset from a base that
  // lives in the kernel's constant bank
  const char* srcq[27];
  char* dstq[27];
  // K_PULL and K_AA_ODD sweeps of fully periodic domains: the stream each
  // direction q reads from (AA odd: slot qbar), shifted by the neighbour
  // offset -(c_qx + nx c_qy + nx ny c_qz) cells, and (AA odd) the stream it
  // writes to, shifted by +(...).  A cell whose y and z neighbours do not
  // wrap then reaches every neighbour with one cell offset (plus a per-thread
  // x wrap), as the AA even sweep does.
  const char* srci[27];
  char* dsti[27];
  // masked domains: fluid cells in ascending order as (cell index, link-mask
  // word) pairs, n_main without wrapped neighbour accesses followed by n_wrap
  // with; the mask word is zero when a separate boundary kernel resolves the
  // boundary links
  const uint2* list;
  int n_main, n_wrap;
  int boundary_mode;  // LBM_BOUNDARY_SEPARATE: the sweep streams every link as fluid
  int special_wrap;   // list builder: cells with inlet/outlet links go to the second launch
  int list_ahead;     // main list launch: distance, in entries, of the L2 prefetch of entries
  int pop_ahead;      // AA list launches (32-bit light operators), FP16 two-cell AA even launch:
                      // distance, in entries or cells, of the L2 prefetch of populations
  // masked sweeps: element offsets, relative to the cell and to the stream of
  // the lower slot of the pair (q, qbar), of the population direction q
  // reads (lf: fluid link, lb: boundary link) and writes (sf, sb: fluid or
  // boundary link (x, qbar)); unsigned, added modulo 2^32
  unsigned lf[27], lb[27], sf[27], sb[27];
  // bounds-checking build (LBM_DEBUG_BOUNDS): bytes of each population array
  // and the device word that records an access outside src or dst
  size_t pdf_bytes;
  unsigned* bounds_flag;
};

// Every population access of the sweep kernels goes through pdf_ld/pdf_st.
// Built with LBM_DEBUG_BOUNDS they check the address against the src and dst
// arrays and, outside both, record it in *bounds_flag and skip the access
// (a load returns zero) instead of trapping; the synchronising calls of the
// API then return LBM_E_BOUNDS.  Otherwise they are plain accesses.
template <class V>
__device__ __forceinline__ bool pdf_in_bounds(const SweepArgs& a, const void* p) {
  const char* c = static_cast<const char*>(p);
  const char* s = static_cast<const char*>(a.src);
  const char* d = static_cast<const char*>(a.dst);
  const bool in_s = s && c >= s && c + sizeof(V) <= s + a.pdf_bytes;
  const bool in_d = d && c >= d && c + sizeof(V) <= d + a.pdf_bytes;
  return in_s || in_d;
}
template <class V>
__device__ __forceinline__ V pdf_ld(const SweepArgs& a, const void* base, long long idx) {
  const V* p = static_cast<const V*>(base) + idx;
#ifdef LBM_DEBUG_BOUNDS
  if (!pdf_in_bounds<V>(a, p)) {
    atomicOr(a.bounds_flag, 1u);
    return V();
  }
#endif
  return *p;
}
template <class V>
__device__ __forceinline__ void pdf_st(const SweepArgs& a, void* base, long long idx, V v) {
  V* p = static_cast<V*>(base) + idx;
#ifdef LBM_DEBUG_BOUNDS
  if (!pdf_in_bounds<V>(a, p)) {
    atomicOr(a.bounds_flag, 1u);
    return;
  }
#endif
  *p = v;
}

constexpr int kBlockX = 128;

// cell offsets of the 3x3x3 neighbourhood, periodic wrap (non-periodic
// out-of-range neighbours are never dereferenced: their links are masked)
struct Nbr {
  int xo[3], yo[3], zo[3];
  __device__ __forceinline__ int at(int dx, int dy, int dz) const { return xo[dx + 1] + yo[dy + 1] + zo[dz + 1]; }
};

__device__ __forceinline__ Nbr make_nbr(const Geom& g, int x, int y, int z) {
  Nbr n;
  n.xo[0] = x == 0 ? g.nx - 1 : x - 1;
  n.xo[1] = x;
  n.xo[2] = x == g.nx - 1 ? 0 : x + 1;
  const int sy = g.nx;
  n.yo[0] = (y == 0 ? g.ny - 1 : y - 1) * sy;
  n.yo[1] = y * sy;
  n.yo[2] = (y == g.ny - 1 ? 0 : y + 1) * sy;
  const int sz = g.nx * g.ny;
  n.zo[0] = (z == 0 ? g.nz - 1 : z - 1) * sz;
  n.zo[1] = z * sz;
  n.zo[2] = (z == g.nz - 1 ? 0 : z + 1) * sz;
  return n;
}

// True when the y and z neighbours of row (y, z) lie inside the box without
// wrapping (1 <= y <= ny - 2 and, in 3-D, 1 <= z <= nz - 2).
template <class L>
__device__ __forceinline__ bool row_inner(const Geom& g, int y, int z) {
  const bool iy = unsigned(y - 1) < unsigned(g.ny - 2);
  if constexpr (L::D == 2) return iy;
  else return iy && unsigned(z - 1) < unsigned(g.nz - 2);
}

// The same for the esoteric twist, which only touches positive neighbours
// (y <= ny - 2 and, in 3-D, z <= nz - 2).
template <class L>
__device__ __forceinline__ bool row_inner_eso(const Geom& g, int y, int z) {
  const bool iy = unsigned(y) < unsigned(g.ny - 1);
  if constexpr (L::D == 2) return iy;
  else return iy && unsigned(z) < unsigned(g.nz - 1);
}

// Boundary type of the link whose source cell is (sx, sy, sz) (may lie one
// cell outside the box).  Arguments are passed by value so that the rare
// call never takes the address of the kernel's parameter block.
static __device__ __noinline__ int link_type(const uint8_t* flags, int nx, int ny, int nz, int per_bits, int sx, int sy,
                                      int sz) {
  if (sx < 0 || sx >= nx) { if (!(per_bits & 1)) return L_NOSLIP; sx = (sx + nx) % nx; }
  if (sy < 0 || sy >= ny) { if (!(per_bits & 2)) return L_NOSLIP; sy = (sy + ny) % ny; }
  if (sz < 0 || sz >= nz) { if (!(per_bits & 4)) return L_NOSLIP; sz = (sz + nz) % nz; }
  if (flags == nullptr) return L_NOSLIP;
  return link_type_of_flag(flags[sx + nx * (sy + ny * sz)]);
}

__device__ __forceinline__ int per_bits(const Geom& g) {
  return (g.per[0] ? 1 : 0) | (g.per[1] ? 2 : 0) | (g.per[2] ? 4 : 0);
}

#define LBM_LINK_TYPE(a, sx, sy, sz) \
  link_type((a).flags, (a).g.nx, (a).g.ny, (a).g.nz, per_bits((a).g), (sx), (sy), (sz))

// Parameters of the outlet condition, copied out of the kernel arguments.
struct OutletP {
  double F[3];
  double rho_out;
  int has_force;
  int incompressible;
};

__device__ __forceinline__ OutletP outlet_params(const CollideParams& p) {
  OutletP o;
  o.F[0] = p.F[0]; o.F[1] = p.F[1]; o.F[2] = p.F[2];
  o.rho_out = p.rho_out;
  o.has_force = p.has_force;
  o.incompressible = p.incompressible;
  return o;
}

template <class L, class T>
__device__ __forceinline__ T ubb_term(int q, const CollideParams& p) {
  // 2 w_q (c_q . u_w) / c_s^2
  const double cu = L::cx(q) * p.u_wall[0] + L::cy(q) * p.u_wall[1] + L::cz(q) * p.u_wall[2];
  return T(6.0 * L::w(q) * cu);
}

// Value domain of populations in registers: DH = true holds h = f - w (shifted
// storage, MRT, cumulant), DH = false holds f itself (unshifted storage with
// SRT/TRT, which then needs no conversion at all).
template <class ST, bool DH>
struct Dom {
  using T = typename ST::T;
  using S = typename ST::S;
  __device__ static __forceinline__ T load(S s, double w) {
    if constexpr (DH) return ST::to_h(s, w);
    else return T(s);
  }
  __device__ static __forceinline__ S store(T v, double w) {
    if constexpr (DH) return ST::from_h(v, w);
    else return S(v);
  }
};

template <class ST, int OP>
constexpr bool dom_h() {
  return ST::shifted || !(OP == OP_SRT || OP == OP_TRT || OP == OP_SRT_LES || OP == OP_TRT_LES);
}

// Outlet value f^eq_q(rho_out, u) in the register domain (minus w_q if DH).
template <class L, class T, bool DH>
__device__ __forceinline__ T outlet_value(int q, const T (&u)[3], const OutletP& p) {
  const T rho = T(p.rho_out);
  const T rho0 = p.incompressible ? T(1) : rho;
  const T cu = T(L::cx(q)) * u[0] + T(L::cy(q)) * u[1] + T(L::cz(q)) * u[2];
  const T usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T feq_dev = T(L::w(q)) * ((rho - T(1)) + rho0 * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
  return DH ? feq_dev : feq_dev + T(L::w(q));
}

// Velocity of post-collision populations: (sum c P - F/2) / rho_0(P).
template <class L, class T, bool DH>
__device__ __forceinline__ void post_velocity(const T (&v)[L::Q], const OutletP& p, T (&u)[3]) {
  T r = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    r += v[q];
    j[0] += T(L::cx(q)) * v[q];
    j[1] += T(L::cy(q)) * v[q];
    j[2] += T(L::cz(q)) * v[q];
  }
  if (p.has_force) {
    j[0] -= T(0.5 * p.F[0]); j[1] -= T(0.5 * p.F[1]); j[2] -= T(0.5 * p.F[2]);
  }
  const T rho = DH ? T(1) + r : r;
  const T inv = T(1) / (p.incompressible ? T(1) : rho);
  u[0] = j[0] * inv; u[1] = j[1] * inv; u[2] = L::D == 3 ? j[2] * inv : T(0);
}

// Value of an inlet or outlet pull link (x, q) whose no-slip value v_noslip
// = P_qbar(x) has already been loaded.  Rare path (cells next to an inlet or
// outlet), so it is not inlined.  The outlet value needs u_P(x), the
// velocity of the cell's P: the first outlet link of a cell loads and
// reduces P(x) into up and sets have_up, and the cell's other outlet links
// reuse it (the caller starts each cell with have_up = 0).
template <class L, class ST, bool DH>
__device__ __noinline__ typename ST::T pull_special(const typename ST::S* src, long long N, int cell, int q, int type,
                                                    typename ST::T v_noslip, const OutletP p, double ubb,
                                                    typename ST::T (&up)[3], int& have_up) {
  using T = typename ST::T;
  if (type == L_INLET) return v_noslip + T(ubb);
  if (type != L_OUTLET) return v_noslip;
  if (!have_up) {
    T v[L::Q];
#pragma unroll
    for (int k = 0; k < L::Q; ++k) v[k] = Dom<ST, DH>::load(src[k * N + cell], L::w(k));
    post_velocity<L, T, DH>(v, p, up);
    have_up = 1;
  }
  return outlet_value<L, T, DH>(q, up, p);
}

template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p, std::integral_constant<int, OP_SRT>) {
  collide_pairs<L, T, OP_SRT, DH>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p, std::integral_constant<int, OP_TRT>) {
  collide_pairs<L, T, OP_TRT, DH>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p,
                                        std::integral_constant<int, OP_SRT_LES>) {
  collide_pairs<L, T, OP_SRT_LES, DH>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p,
                                        std::integral_constant<int, OP_TRT_LES>) {
  collide_pairs<L, T, OP_TRT_LES, DH>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p, std::integral_constant<int, OP_MRT>) {
  static_assert(DH, "MRT works on shifted populations");
  collide_mrt<L, T>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p, std::integral_constant<int, OP_MRT3>) {
  static_assert(DH, "MRT works on shifted populations");
  collide_mrt3<L, T>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p, std::integral_constant<int, OP_KBC>) {
  static_assert(DH, "KBC works on shifted populations");
  collide_kbc<L, T>(v, p);
}
template <class L, class T, bool DH>
__device__ __forceinline__ void collide(T (&v)[L::Q], const CollideParams& p, std::integral_constant<int, OP_CUM>) {
  static_assert(DH, "the cumulant operator works on shifted populations");
  if constexpr (L::Q == 27) collide_cumulant<T>(v, p);
}

// ------------------------------------------------------------------- sweep
// The light operators (SRT, TRT, their Smagorinsky variants, MRT with one
// higher-order rate) in 32-bit arithmetic fit 56 registers: their kernels are
// compiled for 9 resident blocks of 128 threads (36 warps) per SM, so that
// the rarely used Guo-force branch cannot push the common path past that.
// The other operators keep the compiler's own register choice.
constexpr int kLightBlocks = 9;
template <class ST, int OP>
constexpr bool light_op() {
  return (OP == OP_SRT || OP == OP_TRT || OP == OP_SRT_LES || OP == OP_TRT_LES || OP == OP_MRT3) &&
         sizeof(typename ST::T) == 4;
}

// Fully periodic domains without flags: one thread per cell, 128-thread
// blocks along x, grid (nx/128, ny, nz).
template <class L, class ST, int OP, int KIND>
__device__ __forceinline__ void sweep_dense(const SweepArgs& a) {
  using T = typename ST::T;
  using S = typename ST::S;
  constexpr bool DH = dom_h<ST, OP>();
  using D = Dom<ST, DH>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int cell = x + a.g.nx * (y + a.g.ny * z);
  const Nbr nb = make_nbr(a.g, x, y, z);
  T v[L::Q];
  // rows away from the y and z faces (uniform per block) use the shifted
  // stream bases with a per-thread x wrap
  constexpr bool ESO = KIND == K_ESO_EVEN || KIND == K_ESO_ODD;
  bool fast = false;
  if constexpr (ESO) fast = row_inner_eso<L>(a.g, y, z);
  else if constexpr (KIND != K_AA_EVEN) fast = row_inner<L>(a.g, y, z);

  if constexpr (ESO) {
    if (fast) {
      const int ip = cell - (x == a.g.nx - 1 ? a.g.nx : 0);  // location x + 1 with the x wrap
#pragma unroll
      for (int q = 0; q < L::Q; ++q)
        v[q] = D::load(pdf_ld<S>(a, a.srci[q], eso_rd(L::cx(q)) ? ip : cell), L::w(q));
    } else {
#pragma unroll
      for (int q = 0; q < L::Q; ++q) {
        const int qs = KIND == K_ESO_EVEN ? q : opp(q);
        const int idx = nb.at(eso_rd(L::cx(q)), eso_rd(L::cy(q)), eso_rd(L::cz(q)));
        v[q] = D::load(pdf_ld<S>(a, a.srcq[qs], idx), L::w(q));
      }
    }
  } else if constexpr (KIND == K_AA_EVEN) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) v[q] = D::load(pdf_ld<S>(a, a.srcq[q], cell), L::w(q));
  } else if (fast) {
    // x - c_q with the x wrap: c_x = +1 reads x - 1 (wraps at x = 0), c_x = -1 reads x + 1
    const int im = cell + (x == 0 ? a.g.nx : 0);
    const int ip = cell - (x == a.g.nx - 1 ? a.g.nx : 0);
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      const int idx = L::cx(q) > 0 ? im : (L::cx(q) < 0 ? ip : cell);
      v[q] = D::load(pdf_ld<S>(a, a.srci[q], idx), L::w(q));
    }
  } else {
    // pull: P_q(x - c_q) = src[q][x - c_q];  AA odd: A[qbar][x - c_q]
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      const int qs = KIND == K_PULL ? q : opp(q);
      v[q] = D::load(pdf_ld<S>(a, a.srcq[qs], nb.at(-L::cx(q), -L::cy(q), -L::cz(q))), L::w(q));
    }
  }

  collide<L, T, DH>(v, a.cp, std::integral_constant<int, OP>{});

  if constexpr (KIND == K_PULL) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) pdf_st<S>(a, a.dstq[q], cell, D::store(v[q], L::w(q)));
  } else if constexpr (KIND == K_AA_EVEN) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) pdf_st<S>(a, a.dstq[opp(q)], cell, D::store(v[q], L::w(q)));
  } else {
    // The store offsets are rebuilt from a fresh read of %tid.x: an asm with
    // side effects is not moved above the loads and its result cannot be
    // merged with the offsets of the load phase, so the offsets are not held
    // in registers across the collision.
    int tx;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tx));
    const int xs = blockIdx.x * blockDim.x + tx;
    const int cs = xs + a.g.nx * (y + a.g.ny * z);
    if (fast) {
      // x + c_q with the x wrap: c_x = +1 writes x + 1 (wraps at nx - 1), c_x = -1 writes x - 1
      const int ip = cs - (xs == a.g.nx - 1 ? a.g.nx : 0);
      const int im = cs + (xs == 0 ? a.g.nx : 0);
#pragma unroll
      for (int q = 0; q < L::Q; ++q) {
        const int idx = ESO ? (eso_wr(L::cx(q)) ? ip : cs) : (L::cx(q) > 0 ? ip : (L::cx(q) < 0 ? im : cs));
        pdf_st<S>(a, a.dsti[q], idx, D::store(v[q], L::w(q)));
      }
    } else {
      const Nbr nbs = make_nbr(a.g, xs, y, z);
#pragma unroll
      for (int q = 0; q < L::Q; ++q) {
        // AA odd: A[q][x + c_q];  esoteric twist: slot qbar (even) or q (odd) at x + max(c_q, 0)
        const int qd = KIND == K_ESO_EVEN ? opp(q) : q;
        const int idx = ESO ? nbs.at(eso_wr(L::cx(q)), eso_wr(L::cy(q)), eso_wr(L::cz(q)))
                            : nbs.at(L::cx(q), L::cy(q), L::cz(q));
        pdf_st<S>(a, a.dstq[qd], idx, D::store(v[q], L::w(q)));
      }
    }
  }
}

template <class L, class ST, int OP, int KIND>
__global__ void __launch_bounds__(kBlockX) k_sweep(const SweepArgs a) {
  sweep_dense<L, ST, OP, KIND>(a);
}
template <class L, class ST, int OP, int KIND>
__global__ void __launch_bounds__(kBlockX, kLightBlocks) k_sweep_light(const SweepArgs a) {
  sweep_dense<L, ST, OP, KIND>(a);
}

__device__ __forceinline__ void cell_coords(const Geom& g, long long cell, int& x, int& y, int& z) {
  x = (int)(cell % g.nx);
  const long long r = cell / g.nx;
  y = (int)(r % g.ny);
  z = (int)(r / g.ny);
}

// ------------------------------------------------------- fluid-cell lists
// Domains with a link mask (flags or a non-periodic axis) are swept over the
// list of their fluid cells in ascending order, so no warp carries lanes of
// solid cells (in a porous channel most warps would).  Each entry packs the
// cell index with its link-mask word, so a thread reaches its populations
// after one coalesced 8-byte load.  The list holds the cells without a
// wrapped neighbour access first (n_main of them) and then the cells on a
// face of a periodic axis (n_wrap), which a second launch sweeps with
// coordinate-based addressing.  A no-slip link only changes which slot is
// read (pull, AA odd) or written (AA odd, esoteric twist), so the address is
// selected without branching; the few cells with an inlet or outlet link
// (LBM_MASK_SPECIAL) take an out-of-line fix-up of those links' values.

// 0: not fluid; 1: no wrapped neighbour access; 2: on a face of a periodic
// axis, or (two-grid pull resolving its boundary links in the sweep) with an
// inlet or outlet link: the pull fixes those values up before the collision,
// which the main launch does not carry
template <class L>
__device__ __forceinline__ int list_category(const SweepArgs& a, long long cell) {
  const uint32_t m = a.mask[cell];
  if (m & MASK_SOLID) return 0;
  if ((m & MASK_SPECIAL) && a.special_wrap) return 2;
  int x, y, z;
  cell_coords(a.g, cell, x, y, z);
  bool wrap = (a.g.per[0] && (x == 0 || x == a.g.nx - 1)) || (a.g.per[1] && (y == 0 || y == a.g.ny - 1));
  if constexpr (L::D == 3) wrap = wrap || (a.g.per[2] && (z == 0 || z == a.g.nz - 1));
  return wrap ? 2 : 1;
}

constexpr int kListThreads = 256;
constexpr int kListChunk = 4 * kListThreads;  // cells per block of the list builder

// counts[b] and counts[nblk + b]: main and wrap cells of chunk b
template <class L>
__global__ void __launch_bounds__(kListThreads) k_list_count(const SweepArgs a, int nblk, int* __restrict__ counts) {
  __shared__ int sm[2];
  if (threadIdx.x < 2) sm[threadIdx.x] = 0;
  __syncthreads();
  int c1 = 0, c2 = 0;
  for (int k = 0; k < 4; ++k) {
    const long long cell = (long long)blockIdx.x * kListChunk + k * kListThreads + threadIdx.x;
    if (cell < a.g.N) {
      const int cat = list_category<L>(a, cell);
      c1 += cat == 1;
      c2 += cat == 2;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sm[0], c1);
    atomicAdd(&sm[1], c2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    counts[blockIdx.x] = sm[0];
    counts[nblk + blockIdx.x] = sm[1];
  }
}

// Writes each chunk's cells at its exclusive offsets (offsets[b] for main
// cells, offsets[nblk + b] for wrap cells, both absolute), in ascending order,
// each as (cell, link-mask word; zero with a separate boundary kernel).
template <class L>
__global__ void __launch_bounds__(kListThreads) k_list_scatter(const SweepArgs a, int nblk,
                                                                const int* __restrict__ offsets, uint2* __restrict__ list) {
  __shared__ int warp_tot[2][kListThreads / 32];
  int base1 = offsets[blockIdx.x], base2 = offsets[nblk + blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 4; ++k) {
    const long long cell = (long long)blockIdx.x * kListChunk + k * kListThreads + threadIdx.x;
    const int cat = cell < a.g.N ? list_category<L>(a, cell) : 0;
    const unsigned m1 = __ballot_sync(0xffffffffu, cat == 1), m2 = __ballot_sync(0xffffffffu, cat == 2);
    const unsigned below = (1u << lane) - 1u;
    if (lane == 0) {
      warp_tot[0][wid] = __popc(m1);
      warp_tot[1][wid] = __popc(m2);
    }
    __syncthreads();
    int pre1 = 0, pre2 = 0, tot1 = 0, tot2 = 0;
    for (int w = 0; w < kListThreads / 32; ++w) {
      if (w < wid) { pre1 += warp_tot[0][w]; pre2 += warp_tot[1][w]; }
      tot1 += warp_tot[0][w];
      tot2 += warp_tot[1][w];
    }
    const unsigned word = (cat != 0 && !a.boundary_mode) ? a.mask[cell] : 0u;
    if (cat == 1) list[base1 + pre1 + __popc(m1 & below)] = make_uint2(unsigned(cell), word);
    if (cat == 2) list[base2 + pre2 + __popc(m2 & below)] = make_uint2(unsigned(cell), word);
    base1 += tot1;
    base2 += tot2;
    __syncthreads();
  }
}

// Entry i of the list, loaded again after the collision: an asm with side
// effects is neither hoisted above the collision nor merged with the first
// load, so neither the entry nor its address stays in registers across it.
__device__ __forceinline__ uint2 reload_entry(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}


// Sweep over list[0, n_main) (WRAP = false: every neighbour access is the
// cell's own index plus a fixed offset) or over list[n_main, n_main + n_wrap)
// (WRAP = true: neighbour indices from the coordinates, with wrapping).
// Inlet and outlet links (x, p = qbar) of a cell swept by a single-array
// pattern on the plain list path: the value B_p(P(x)) replaces the P_q(x)
// the common stores wrote into the link's slot.  v: the cell's
// post-collision populations in the register domain of D.
template <class L, class ST, bool DH, int KIND>
__device__ __forceinline__ void store_special_links(const SweepArgs& a, const typename ST::T (&v)[L::Q], int cs,
                                                    uint32_t ms) {
  using T = typename ST::T;
  using S = typename ST::S;
  using D = Dom<ST, DH>;
  int x, y, z;
  cell_coords(a.g, cs, x, y, z);
  const OutletP op = outlet_params(a.cp);
  T up[3];
  post_velocity<L, T, DH>(v, op, up);
#pragma unroll
  for (int q = 1; q < L::Q; ++q) {
    const int p = opp(q);
    if ((ms >> p) & 1u) {
      const int t = LBM_LINK_TYPE(a, x + L::cx(q), y + L::cy(q), z + L::cz(q));
      if (t == L_INLET || t == L_OUTLET) {
        const T val = t == L_INLET ? v[q] + ubb_term<L, T>(p, a.cp) : outlet_value<L, T, DH>(p, up, op);
        if constexpr (KIND == K_AA_EVEN) {
          pdf_st<S>(a, a.dstq[p], cs, D::store(val, L::w(q)));
        } else {
          const int lo = q < p ? q : p;
          pdf_st<S>(a, a.dstq[lo], unsigned(cs) + a.sb[q], D::store(val, L::w(q)));
        }
      }
    }
  }
}

// One list entry (cell, link-mask word) at list position i.
template <class L, class ST, int OP, int KIND, bool WRAP>
__device__ __forceinline__ void sweep_list(const SweepArgs& a, const uint2 entry, const int i) {
  using T = typename ST::T;
  using S = typename ST::S;
  constexpr bool DH = dom_h<ST, OP>();
  using D = Dom<ST, DH>;
  constexpr bool ESO = KIND == K_ESO_EVEN || KIND == K_ESO_ODD;
  const int cell = int(entry.x);
  const uint32_t mask = entry.y;
  T v[L::Q];
  if constexpr (WRAP) {
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    const Nbr nb = make_nbr(a.g, x, y, z);
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      // pull:   fluid source -> src[q][x - c_q];  boundary -> src[qbar][x]
      // AA odd: fluid source -> A[qbar][x - c_q]; boundary -> A[q][x]
      // esoteric twist: slot q (even) or qbar (odd) at x + max(-c_q, 0)
      const bool b = (mask >> q) & 1u;
      int qs, idx;
      if constexpr (ESO) {
        qs = KIND == K_ESO_EVEN ? q : opp(q);
        idx = nb.at(eso_rd(L::cx(q)), eso_rd(L::cy(q)), eso_rd(L::cz(q)));
      } else if constexpr (KIND == K_AA_EVEN) {
        qs = q;
        idx = cell;
      } else {
        qs = KIND == K_PULL ? (b ? opp(q) : q) : (b ? q : opp(q));
        idx = b ? cell : nb.at(-L::cx(q), -L::cy(q), -L::cz(q));
      }
      v[q] = D::load(pdf_ld<S>(a, a.srcq[qs], idx), L::w(q));
    }
  } else {
    // The two slots a direction can touch, q and qbar, are adjacent streams:
    // one base (the lower slot) plus a per-direction offset from the kernel
    // arguments, selected by the boundary bit (the element index stays below
    // 2 N - 1 < 2^32)
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      const bool b = (mask >> q) & 1u;
      if constexpr (ESO) {
        v[q] = D::load(pdf_ld<S>(a, a.srci[q], cell), L::w(q));
      } else if constexpr (KIND == K_AA_EVEN) {
        v[q] = D::load(pdf_ld<S>(a, a.srcq[q], cell), L::w(q));
      } else {
        // pull: fluid src[q][x - c_q], boundary src[qbar][x];
        // AA odd: fluid A[qbar][x - c_q], boundary A[q][x]
        const int lo = q < opp(q) ? q : opp(q);
        const unsigned idx = unsigned(cell) + (b ? a.lb[q] : a.lf[q]);
        v[q] = D::load(pdf_ld<S>(a, a.srcq[lo], idx), L::w(q));
      }
    }
  }
  if constexpr (KIND == K_PULL && WRAP) {
    if (mask & MASK_SPECIAL) {
      int x, y, z;
      cell_coords(a.g, cell, x, y, z);
      const OutletP op = outlet_params(a.cp);
      T up[3];
      int have_up = 0;
      for (int q = 1; q < L::Q; ++q) {
        if ((mask >> q) & 1u) {
          const int t = LBM_LINK_TYPE(a, x - L::cx(q), y - L::cy(q), z - L::cz(q));
          const double ubb = 6.0 * L::w(q) * (L::cx(q) * a.cp.u_wall[0] + L::cy(q) * a.cp.u_wall[1] +
                                              L::cz(q) * a.cp.u_wall[2]);
          v[q] = pull_special<L, ST, DH>(static_cast<const S*>(a.src), a.g.N, cell, q, t, v[q], op, ubb, up,
                                         have_up);
        }
      }
    }
  }

  collide<L, T, DH>(v, a.cp, std::integral_constant<int, OP>{});

  if constexpr (KIND != K_PULL && WRAP) {
    // inlet/outlet links (x, p = qbar): the value written for direction q is
    // B_p(P(x)) instead of P_q(x); no-slip links keep P_q(x) = B_p(P(x))
    if (mask & MASK_SPECIAL) {
      int x, y, z;
      cell_coords(a.g, cell, x, y, z);
      const OutletP op = outlet_params(a.cp);
      T up[3];
      post_velocity<L, T, DH>(v, op, up);
#pragma unroll
      for (int q = 1; q < L::Q; ++q) {
        const int p = opp(q);
        if ((mask >> p) & 1u) {
          const int t = LBM_LINK_TYPE(a, x + L::cx(q), y + L::cy(q), z + L::cz(q));
          if (t == L_INLET) v[q] += ubb_term<L, T>(p, a.cp);
          else if (t == L_OUTLET) v[q] = outlet_value<L, T, DH>(p, up, op);
        }
      }
    }
  }
  if constexpr (KIND == K_PULL) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) pdf_st<S>(a, a.dstq[q], cell, D::store(v[q], L::w(q)));
  } else if constexpr (KIND == K_AA_EVEN) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) pdf_st<S>(a, a.dstq[opp(q)], cell, D::store(v[q], L::w(q)));
  } else if constexpr (WRAP) {
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    const Nbr nbs = make_nbr(a.g, x, y, z);
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      // AA odd: fluid destination -> A[q][x + c_q]; boundary link (x, qbar) -> A[qbar][x]
      // esoteric twist: slot qbar (even) or q (odd) at x + max(c_q, 0); a
      // boundary link (x, qbar) takes the other slot
      const int p = opp(q);
      const bool b = (mask >> p) & 1u;
      int qd, idx;
      if constexpr (ESO) {
        qd = ((KIND == K_ESO_EVEN) != b) ? p : q;
        idx = nbs.at(eso_wr(L::cx(q)), eso_wr(L::cy(q)), eso_wr(L::cz(q)));
      } else {
        qd = b ? p : q;
        idx = b ? cell : nbs.at(L::cx(q), L::cy(q), L::cz(q));
      }
      pdf_st<S>(a, a.dstq[qd], idx, D::store(v[q], L::w(q)));
    }
  } else {
    // the entry is read again (a cache hit) rather than held across the
    // collision
    const uint2 es = reload_entry(a.list + i);
    const int cs = int(es.x);
    const uint32_t ms = es.y;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      // AA odd: fluid A[q][x + c_q], boundary link (x, qbar) A[qbar][x];
      // esoteric twist: slot qbar (even) or q (odd) at x + max(c_q, 0), a
      // boundary link takes the other slot of the same location
      const int p = opp(q);
      const bool b = (ms >> p) & 1u;
      const int lo = q < p ? q : p;
      const unsigned idx = unsigned(cs) + (b ? a.sb[q] : a.sf[q]);
      pdf_st<S>(a, a.dstq[lo], idx, D::store(v[q], L::w(q)));
    }
  }
  if constexpr (KIND != K_PULL && !WRAP) {
    // Cells with inlet or outlet links (single-array patterns): every link
    // was stored above as if it were a no-slip link (B_p(P(x)) = P_q(x) for
    // p = qbar); the inlet and outlet ones are stored again with their own
    // value B_p(P(x)) into the same slot.  After the stores, so that the
    // common path carries none of this.
    const uint2 es = reload_entry(a.list + i);
    if (es.y & MASK_SPECIAL) store_special_links<L, ST, DH, KIND>(a, v, int(es.x), es.y);
  }
}

// AA list sweeps of the light operators with 32-bit storage also prefetch
// populations (below).  Measured on the porous D3Q19 MRT channel (FP32, one
// GB300): even step 0.228 -> 0.203 ms, odd step 0.268 -> 0.224 ms.  In the
// two-grid pull it cost 4 %, and with 16-bit storage, whose sweep is issue
// bound, 7 %; those sweeps carry no prefetch code.
template <class L, class ST, int OP>
constexpr bool list_pop_prefetch() {
  return sizeof(typename ST::S) == 4 && light_op<ST, OP>();
}

// Main list launch, one entry per thread.  Each thread first asks the L2 to
// fetch the entry that a block about one and a half resident grids later
// will need (SweepArgs::list_ahead entries ahead), so that by the time that
// block starts, its dependent entry load hits the L2 instead of DRAM; the
// prefetch holds no register and nothing waits for it.  In the AA steps of
// list_pop_prefetch() operators the thread also prefetches the q
// populations of the cell SweepArgs::pop_ahead entries ahead (a third of a
// resident grid: that entry is already in the L2), so that the block that
// sweeps it finds them in the L2: the addresses that cell's loads will use
// (even step: its own slots; odd step: the slots its links read, at the
// neighbour for a fluid link and at the cell for a boundary link).
template <class L, class ST, int OP, int KIND>
__device__ __forceinline__ void sweep_list_main(const SweepArgs& a) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned ahead = i + unsigned(a.list_ahead);  // n_main < 2^31, list_ahead < 2^30: no wrap
  if ((threadIdx.x & 15) == 0 && ahead < unsigned(a.n_main))
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.list + ahead));
  if constexpr ((KIND == K_AA_EVEN || KIND == K_AA_ODD) && list_pop_prefetch<L, ST, OP>()) {
    if (a.pop_ahead > 0) {
      const unsigned pi = i + unsigned(a.pop_ahead);  // pop_ahead < list_ahead: no wrap
      if (pi < unsigned(a.n_main)) {
        const uint2 pe = a.list[pi];
        using S = typename ST::S;
#pragma unroll
        for (int q = 0; q < L::Q; ++q) {
          const char* p;
          if constexpr (KIND == K_AA_EVEN) {
            p = a.srcq[q] + size_t(pe.x) * sizeof(S);
          } else {
            const bool b = (pe.y >> q) & 1u;
            const int lo = q < opp(q) ? q : opp(q);
            p = a.srcq[lo] + size_t(unsigned(pe.x) + (b ? a.lb[q] : a.lf[q])) * sizeof(S);
          }
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        }
      }
    }
  }
  if (i < unsigned(a.n_main)) sweep_list<L, ST, OP, KIND, false>(a, a.list[i], int(i));
}

template <class L, class ST, int OP, int KIND>
__global__ void __launch_bounds__(kBlockX) k_sweep_list(const SweepArgs a) {
  sweep_list_main<L, ST, OP, KIND>(a);
}
template <class L, class ST, int OP, int KIND>
__global__ void __launch_bounds__(kBlockX, kLightBlocks) k_sweep_list_light(const SweepArgs a) {
  sweep_list_main<L, ST, OP, KIND>(a);
}

// The main list sweep of D3Q19 with 16-bit storage under SRT, TRT and
// one-higher-rate MRT, with a register cap.  Each thread waits on two
// dependent loads (list entry, then link mask) before its population loads
// can issue, and with 2-byte populations it moves half the bytes per load,
// so it needs more warps in flight per SM than the 32-bit sweep to keep the
// bytes in flight that hide the latency; the cap trades a few values spilled
// to L1 for those warps (with 32-bit storage the same cap was slower).
#ifndef LBM_LIST_MAXNREG
#define LBM_LIST_MAXNREG 48
#endif

template <class L, class ST, int OP>
constexpr bool list_capped() {
  return L::Q == 19 && sizeof(typename ST::S) == 2 && (OP == OP_SRT || OP == OP_TRT || OP == OP_MRT3);
}

template <class L, class ST, int OP, int KIND>
__global__ void __maxnreg__(LBM_LIST_MAXNREG) k_sweep_list_capped(const SweepArgs a) {
  sweep_list_main<L, ST, OP, KIND>(a);
}

template <class L, class ST, int OP, int KIND>
__global__ void __launch_bounds__(kBlockX) k_sweep_list_wrap(const SweepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n_wrap) sweep_list<L, ST, OP, KIND, true>(a, a.list[a.n_main + i], a.n_main + i);
}

// Separate boundary kernel of the two-grid pull (LBM_BOUNDARY_SEPARATE):
// for every boundary link (x, q) of a fluid cell it writes B_q(P(x)) into
// slot q of the link's source cell x - c_q (inside the box, non-fluid), so
// that the following sweep can stream the link like a fluid one.  Each such
// slot belongs to one link; fluid cells' slots are only read.
template <class L, class ST>
__global__ void __launch_bounds__(kBlockX) k_boundary_pull(const SweepArgs a, typename ST::S* __restrict__ P) {
  using T = typename ST::T;
  using S = typename ST::S;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_main + a.n_wrap) return;
  const int cell = int(a.list[i].x);
  const uint32_t mask = a.mask[cell];  // the list's mask words are zero in this mode
  if ((mask & ((1u << L::Q) - 2u)) == 0) return;
  int x, y, z;
  cell_coords(a.g, cell, x, y, z);
  constexpr bool DH = ST::shifted;  // the storage's own value domain
  using D = Dom<ST, DH>;
  const long long N = a.g.N;
  if (!(mask & MASK_SPECIAL)) {
    // no inlet or outlet link: every boundary link is a no-slip copy
    const Nbr nb = make_nbr(a.g, x, y, z);
#pragma unroll
    for (int q = 1; q < L::Q; ++q)
      if ((mask >> q) & 1u)
        pdf_st<S>(a, P, q * N + nb.at(-L::cx(q), -L::cy(q), -L::cz(q)), pdf_ld<S>(a, P, opp(q) * N + cell));
    return;
  }
  T up[3] = {T(0), T(0), T(0)};
  {
    T v[L::Q];
#pragma unroll
    for (int k = 0; k < L::Q; ++k) v[k] = D::load(pdf_ld<S>(a, P, k * N + cell), L::w(k));
    post_velocity<L, T, DH>(v, outlet_params(a.cp), up);
  }
  const Nbr nb = make_nbr(a.g, x, y, z);
#pragma unroll
  for (int q = 1; q < L::Q; ++q) {
    if (!((mask >> q) & 1u)) continue;
    const int t = LBM_LINK_TYPE(a, x - L::cx(q), y - L::cy(q), z - L::cz(q));
    const long long slot = q * N + nb.at(-L::cx(q), -L::cy(q), -L::cz(q));
    const S own = pdf_ld<S>(a, P, opp(q) * N + cell);
    if (t == L_OUTLET) pdf_st<S>(a, P, slot, D::store(outlet_value<L, T, DH>(q, up, outlet_params(a.cp)), L::w(q)));
    else if (t == L_INLET) pdf_st<S>(a, P, slot, D::store(D::load(own, L::w(q)) + ubb_term<L, T>(q, a.cp), L::w(q)));
    else pdf_st<S>(a, P, slot, own);  // no-slip: the stored value itself
  }
}

// ---------------------------------------------------- FP16 two-cell sweep
// Periodic FP16-shifted sweeps with two cells (x0, x0 + 1) per thread.  A
// 2-byte population leaves a warp request at 64 B, so one cell per thread
// keeps too few bytes in flight; here the two cells' populations of each
// direction sit packed in one __half2 register, directions with c_x = 0 move
// both cells with one aligned 32-bit access, the others with two 16-bit
// accesses.  Each cell is unpacked, collided and repacked in turn, so the
// register cost is one packed register per direction plus one collision.
// Requires an even nx (x0 and every row start are then 4-byte aligned).
template <class L, int OP, int KIND>
__global__ void __launch_bounds__(kBlockX) k_sweep_h2(const SweepArgs a) {
  using T = float;
  const int tp = blockIdx.x * blockDim.x + threadIdx.x;
  const int x0 = 2 * tp;
  if (x0 >= a.g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int cell = x0 + a.g.nx * (y + a.g.ny * z);
  const int nx = a.g.nx;
  const int sy = nx, sz = nx * a.g.ny;
  const int yo[3] = {(y == 0 ? a.g.ny - 1 : y - 1) * sy, y * sy, (y == a.g.ny - 1 ? 0 : y + 1) * sy};
  const int zo[3] = {(z == 0 ? a.g.nz - 1 : z - 1) * sz, z * sz, (z == a.g.nz - 1 ? 0 : z + 1) * sz};
  // x of the neighbours of cell 0 (x0) and cell 1 (x0 + 1) for dx = -1, 0, 1
  const int xa[3] = {x0 == 0 ? nx - 1 : x0 - 1, x0, x0 + 1};
  const int xb[3] = {x0, x0 + 1, x0 + 2 == nx ? 0 : x0 + 2};
  constexpr bool ESO = KIND == K_ESO_EVEN || KIND == K_ESO_ODD;
  if constexpr (KIND == K_AA_EVEN) {
    // the even step reads the cell pair's own slots; ask the L2 for those of
    // the pair SweepArgs::pop_ahead cells ahead (a third of a resident grid:
    // blocks start in cell order), which a later block will load.  Measured
    // at 256^3 TRT: even step 0.213 -> 0.195 ms; in the odd step, the pull
    // and the esoteric twist the same prefetch cost 4-17 %, so they carry none.
    const long long pc = (long long)cell + a.pop_ahead;
    if (a.pop_ahead > 0 && pc + 1 < a.g.N) {
#pragma unroll
      for (int q = 0; q < L::Q; ++q)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const __half*>(a.srcq[q]) + pc));
    }
  }
  __half2 P[L::Q];
  // rows whose y/z neighbours do not wrap read through the pre-shifted bases
  // (SweepArgs::srci): the two cells' sources are srci[q][cell] and
  // srci[q][cell + 1], up to the x wrap of the first (source x0 - 1 at x0 = 0)
  // or of the second (source x0 + 2 at x0 + 2 = nx)
  // (measured: faster for the esoteric twist, neutral for pull, slower for
  // the AA odd step, which keeps the coordinate addressing)
  bool fast = false;
  if constexpr (ESO) fast = row_inner_eso<L>(a.g, y, z);
  else if constexpr (KIND == K_PULL) fast = row_inner<L>(a.g, y, z);
  if (fast) {
    const int wa = x0 == 0 ? nx : 0, wb = x0 + 2 == nx ? nx : 0;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      const __half* base = reinterpret_cast<const __half*>(a.srci[q]);
      // does cell 0 read x0 - 1 (+1 direction of pull/AA) / cell 1 read x0 + 2?
      const bool lo = ESO ? false : L::cx(q) > 0;
      const bool hi = ESO ? eso_rd(L::cx(q)) != 0 : L::cx(q) < 0;
      if (!lo && !hi) P[q] = pdf_ld<__half2>(a, base + cell, 0);
      else
        P[q] = __halves2half2(pdf_ld<__half>(a, base, cell + (lo ? wa : 0)),
                              pdf_ld<__half>(a, base, cell + 1 - (hi ? wb : 0)));
    }
  }
  if (!fast) {
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    // pull / AA even / esoteric twist even read slot q; AA odd and esoteric
    // twist odd read slot qbar
    const int qs = (KIND == K_AA_ODD || KIND == K_ESO_ODD) ? opp(q) : q;
    const __half* base = reinterpret_cast<const __half*>(a.srcq[qs]);
    if constexpr (KIND == K_AA_EVEN) {
      P[q] = pdf_ld<__half2>(a, base + cell, 0);
    } else if constexpr (ESO) {
      // location x + max(-c_q, 0): x0 and x0 + 1, or x0 + 1 and x0 + 2
      const int row = yo[eso_rd(L::cy(q)) + 1] + zo[eso_rd(L::cz(q)) + 1];
      if (eso_rd(L::cx(q)) == 0) P[q] = pdf_ld<__half2>(a, base + row + x0, 0);
      else P[q] = __halves2half2(pdf_ld<__half>(a, base, row + xb[1]), pdf_ld<__half>(a, base, row + xb[2]));
    } else {
      const int dx = -L::cx(q), dy = -L::cy(q), dz = -L::cz(q);
      const int row = yo[dy + 1] + zo[dz + 1];
      if (dx == 0) P[q] = pdf_ld<__half2>(a, base + row + x0, 0);
      else P[q] = __halves2half2(pdf_ld<__half>(a, base, row + xa[dx + 1]), pdf_ld<__half>(a, base, row + xb[dx + 1]));
    }
  }
  }
  T v[L::Q];
#pragma unroll
  for (int q = 0; q < L::Q; ++q) v[q] = __low2float(P[q]);
  collide<L, T, true>(v, a.cp, std::integral_constant<int, OP>{});
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    P[q] = __halves2half2(__float2half_rn(v[q]), __high2half(P[q]));
    v[q] = __high2float(P[q]);
  }
  collide<L, T, true>(v, a.cp, std::integral_constant<int, OP>{});
#pragma unroll
  for (int q = 0; q < L::Q; ++q) P[q] = __halves2half2(__low2half(P[q]), __float2half_rn(v[q]));
  if constexpr (KIND == K_PULL) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) pdf_st<__half2>(a, reinterpret_cast<__half*>(a.dstq[q]) + cell, 0, P[q]);
  } else if constexpr (KIND == K_AA_EVEN) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q)
      pdf_st<__half2>(a, reinterpret_cast<__half*>(a.dstq[opp(q)]) + cell, 0, P[q]);
  } else if (fast) {
    // writes through the pre-shifted bases (SweepArgs::dsti): cell 0 writes
    // x0 - 1 (wraps at x0 = 0), cell 1 writes x0 + 2 (wraps at x0 + 2 = nx)
    int tx;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tx));
    const int x1 = 2 * (blockIdx.x * blockDim.x + tx);
    const int c1 = x1 + nx * (y + a.g.ny * z);
    const int wa = x1 == 0 ? nx : 0, wb = x1 + 2 == nx ? nx : 0;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      __half* base = reinterpret_cast<__half*>(a.dsti[q]);
      const bool lo = ESO ? false : L::cx(q) < 0;
      const bool hi = ESO ? eso_wr(L::cx(q)) != 0 : L::cx(q) > 0;
      if (!lo && !hi) {
        pdf_st<__half2>(a, base + c1, 0, P[q]);
      } else {
        pdf_st<__half>(a, base, c1 + (lo ? wa : 0), __low2half(P[q]));
        pdf_st<__half>(a, base, c1 + 1 - (hi ? wb : 0), __high2half(P[q]));
      }
    }
  } else if constexpr (ESO) {
    int tx;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tx));
    const int x1 = 2 * (blockIdx.x * blockDim.x + tx);
    const int yo2[3] = {(y == 0 ? a.g.ny - 1 : y - 1) * sy, y * sy, (y == a.g.ny - 1 ? 0 : y + 1) * sy};
    const int zo2[3] = {(z == 0 ? a.g.nz - 1 : z - 1) * sz, z * sz, (z == a.g.nz - 1 ? 0 : z + 1) * sz};
    const int xb1 = x1 + 1, xb2 = x1 + 2 == nx ? 0 : x1 + 2;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      // slot qbar (even) or q (odd) at x + max(c_q, 0)
      __half* base = reinterpret_cast<__half*>(a.dstq[KIND == K_ESO_EVEN ? opp(q) : q]);
      const int row = yo2[eso_wr(L::cy(q)) + 1] + zo2[eso_wr(L::cz(q)) + 1];
      if (eso_wr(L::cx(q)) == 0) {
        pdf_st<__half2>(a, base + row + x1, 0, P[q]);
      } else {
        pdf_st<__half>(a, base, row + xb1, __low2half(P[q]));
        pdf_st<__half>(a, base, row + xb2, __high2half(P[q]));
      }
    }
  } else {
    // rebuild the neighbour offsets from a fresh %tid.x read (see k_sweep)
    int tx;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tx));
    const int x1 = 2 * (blockIdx.x * blockDim.x + tx);
    const int yo2[3] = {(y == 0 ? a.g.ny - 1 : y - 1) * sy, y * sy, (y == a.g.ny - 1 ? 0 : y + 1) * sy};
    const int zo2[3] = {(z == 0 ? a.g.nz - 1 : z - 1) * sz, z * sz, (z == a.g.nz - 1 ? 0 : z + 1) * sz};
    const int xa2[3] = {x1 == 0 ? nx - 1 : x1 - 1, x1, x1 + 1};
    const int xb2[3] = {x1, x1 + 1, x1 + 2 == nx ? 0 : x1 + 2};
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      __half* base = reinterpret_cast<__half*>(a.dstq[q]);
      const int dx = L::cx(q), dy = L::cy(q), dz = L::cz(q);
      const int row = yo2[dy + 1] + zo2[dz + 1];
      if (dx == 0) {
        pdf_st<__half2>(a, base + row + x1, 0, P[q]);
      } else {
        pdf_st<__half>(a, base, row + xa2[dx + 1], __low2half(P[q]));
        pdf_st<__half>(a, base, row + xb2[dx + 1], __high2half(P[q]));
      }
    }
  }
}

// ------------------------------------------------------------- gather (FP64)
// Populations f(x) of the current time in FP64 (unshifted).
template <class L, class ST>
__device__ void gather_f64(const SweepArgs& a, int view, int x, int y, int z, int cell, uint32_t mask,
                           double (&f)[L::Q]) {
  using S = typename ST::S;
  const S* A = static_cast<const S*>(a.src);
  const long long N = a.g.N;
  const Nbr nb = make_nbr(a.g, x, y, z);
  if (view == V_ESO_EVEN || view == V_ESO_ODD) {
    for (int q = 0; q < L::Q; ++q) {
      const int slot = view == V_ESO_EVEN ? q : opp(q);
      f[q] = ST::to_f64(A[slot * N + nb.at(eso_rd(L::cx(q)), eso_rd(L::cy(q)), eso_rd(L::cz(q)))], L::w(q));
    }
    return;
  }
  if (view == V_AA_NATURAL) {
    for (int q = 0; q < L::Q; ++q) f[q] = ST::to_f64(A[q * N + cell], L::w(q));
    return;
  }
  if (view == V_AA_INVERTED) {
    for (int q = 0; q < L::Q; ++q) {
      if ((mask >> q) & 1u)
        f[q] = ST::to_f64(A[q * N + cell], L::w(q));
      else
        f[q] = ST::to_f64(A[opp(q) * N + nb.at(-L::cx(q), -L::cy(q), -L::cz(q))], L::w(q));
    }
    return;
  }
  // pull: A holds P
  double uP[3] = {0, 0, 0};
  bool have_up = false;
  for (int q = 0; q < L::Q; ++q) {
    if ((mask >> q) & 1u) {
      const int t = LBM_LINK_TYPE(a, x - L::cx(q), y - L::cy(q), z - L::cz(q));
      if (t == L_OUTLET) {
        if (!have_up) {
          double rho = 0, j[3] = {0, 0, 0};
          for (int k = 0; k < L::Q; ++k) {
            const double v = ST::to_f64(A[k * N + cell], L::w(k));
            rho += v;
            j[0] += L::cx(k) * v; j[1] += L::cy(k) * v; j[2] += L::cz(k) * v;
          }
          if (a.cp.has_force) for (int d = 0; d < 3; ++d) j[d] -= 0.5 * a.cp.F[d];
          const double r0 = a.cp.incompressible ? 1.0 : rho;
          for (int d = 0; d < 3; ++d) uP[d] = j[d] / r0;
          if (L::D == 2) uP[2] = 0.0;
          have_up = true;
        }
        const double rho = a.cp.rho_out;
        const double rho0 = a.cp.incompressible ? 1.0 : rho;
        const double cu = L::cx(q) * uP[0] + L::cy(q) * uP[1] + L::cz(q) * uP[2];
        const double usq = uP[0] * uP[0] + uP[1] * uP[1] + uP[2] * uP[2];
        f[q] = L::w(q) * (rho + rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
      } else {
        double v = ST::to_f64(A[opp(q) * N + cell], L::w(q));
        if (t == L_INLET)
          v += 6.0 * L::w(q) * (L::cx(q) * a.cp.u_wall[0] + L::cy(q) * a.cp.u_wall[1] + L::cz(q) * a.cp.u_wall[2]);
        f[q] = v;
      }
    } else {
      f[q] = ST::to_f64(A[q * N + nb.at(-L::cx(q), -L::cy(q), -L::cz(q))], L::w(q));
    }
  }
}

// Shifted populations h = f - w of the current time in the compute type T
// (same views and boundary values as gather_f64).
template <class L, class ST>
__device__ void gather_h(const SweepArgs& a, int view, int x, int y, int z, int cell, uint32_t mask,
                         typename ST::T (&h)[L::Q]) {
  using S = typename ST::S;
  using T = typename ST::T;
  const S* A = static_cast<const S*>(a.src);
  const long long N = a.g.N;
  const Nbr nb = make_nbr(a.g, x, y, z);
  if (view == V_ESO_EVEN || view == V_ESO_ODD) {
    for (int q = 0; q < L::Q; ++q) {
      const int slot = view == V_ESO_EVEN ? q : opp(q);
      h[q] = ST::to_h(A[slot * N + nb.at(eso_rd(L::cx(q)), eso_rd(L::cy(q)), eso_rd(L::cz(q)))], L::w(q));
    }
    return;
  }
  if (view == V_AA_NATURAL) {
    for (int q = 0; q < L::Q; ++q) h[q] = ST::to_h(A[q * N + cell], L::w(q));
    return;
  }
  if (view == V_AA_INVERTED) {
    for (int q = 0; q < L::Q; ++q) {
      if ((mask >> q) & 1u)
        h[q] = ST::to_h(A[q * N + cell], L::w(q));
      else
        h[q] = ST::to_h(A[opp(q) * N + nb.at(-L::cx(q), -L::cy(q), -L::cz(q))], L::w(q));
    }
    return;
  }
  for (int q = 0; q < L::Q; ++q) {
    const bool b = (mask >> q) & 1u;
    h[q] = ST::to_h(A[(b ? opp(q) : q) * N + (b ? cell : nb.at(-L::cx(q), -L::cy(q), -L::cz(q)))], L::w(q));
  }
  if (mask & MASK_SPECIAL) {
    const OutletP op = outlet_params(a.cp);
    T up[3];
    int have_up = 0;
    for (int q = 1; q < L::Q; ++q) {
      if ((mask >> q) & 1u) {
        const int t = LBM_LINK_TYPE(a, x - L::cx(q), y - L::cy(q), z - L::cz(q));
        const double ubb = 6.0 * L::w(q) * (L::cx(q) * a.cp.u_wall[0] + L::cy(q) * a.cp.u_wall[1] +
                                            L::cz(q) * a.cp.u_wall[2]);
        h[q] = pull_special<L, ST, true>(A, N, cell, q, t, h[q], op, ubb, up, have_up);
      }
    }
  }
}

template <class L>
__device__ __forceinline__ void moments_f64(const double (&f)[L::Q], const CollideParams& p, double& rho,
                                            double& rho0, double (&u)[3]) {
  double j[3] = {0, 0, 0};
  rho = 0;
  for (int q = 0; q < L::Q; ++q) {
    rho += f[q];
    j[0] += L::cx(q) * f[q];
    j[1] += L::cy(q) * f[q];
    j[2] += L::cz(q) * f[q];
  }
  if (p.has_force) for (int d = 0; d < 3; ++d) j[d] += 0.5 * p.F[d];
  rho0 = p.incompressible ? 1.0 : rho;
  const double inv = 1.0 / rho0;
  for (int d = 0; d < 3; ++d) u[d] = j[d] * inv;
  if (L::D == 2) u[2] = 0.0;
}

template <class L, class ST>
__global__ void k_populations(const SweepArgs a, int view, double* __restrict__ out) {
  const long long N = a.g.N;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    const uint32_t mask = a.mask ? a.mask[cell] : 0u;
    if (mask & MASK_SOLID) {
      for (int q = 0; q < L::Q; ++q) out[q * N + cell] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    double f[L::Q];
    gather_f64<L, ST>(a, view, x, y, z, (int)cell, mask, f);
    for (int q = 0; q < L::Q; ++q) out[q * N + cell] = f[q];
  }
}

template <class L, class ST, class OUT>
__global__ void k_macroscopic(const SweepArgs a, int view, OUT* __restrict__ rho_out, OUT* __restrict__ u_out) {
  const long long N = a.g.N;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    const uint32_t mask = a.mask ? a.mask[cell] : 0u;
    if (mask & MASK_SOLID) {
      const OUT nan = OUT(__longlong_as_double(0x7ff8000000000000LL));
      rho_out[cell] = nan;
      for (int d = 0; d < L::D; ++d) u_out[d * N + cell] = nan;
      continue;
    }
    using T = typename ST::T;
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    T h[L::Q];
    gather_h<L, ST>(a, view, x, y, z, (int)cell, mask, h);
    T drho = T(0), j[3] = {T(0), T(0), T(0)};
    for (int q = 0; q < L::Q; ++q) {
      drho += h[q];
      j[0] += T(L::cx(q)) * h[q];
      j[1] += T(L::cy(q)) * h[q];
      j[2] += T(L::cz(q)) * h[q];
    }
    if (a.cp.has_force)
      for (int d = 0; d < 3; ++d) j[d] += T(0.5 * a.cp.F[d]);
    const T inv = T(1) / (a.cp.incompressible ? T(1) : T(1) + drho);
    rho_out[cell] = OUT(1.0 + double(drho));
    for (int d = 0; d < L::D; ++d) u_out[d * N + cell] = OUT(j[d] * inv);
  }
}

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// FP64 partial sums (mass, momentum[3], kinetic energy) per block; the
// partials array is caller-provided scratch of gridDim.x * 5 doubles.
template <class L, class ST>
__global__ void __launch_bounds__(kRedThreads) k_reduce_partial(const SweepArgs a, int view, double* partials) {
  const long long N = a.g.N;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    const uint32_t mask = a.mask ? a.mask[cell] : 0u;
    if (mask & MASK_SOLID) continue;
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    double f[L::Q];
    gather_f64<L, ST>(a, view, x, y, z, (int)cell, mask, f);
    double rho, rho0, u[3];
    moments_f64<L>(f, a.cp, rho, rho0, u);
    acc[0] += rho;
    acc[1] += rho0 * u[0];
    acc[2] += rho0 * u[1];
    acc[3] += rho0 * u[2];
    acc[4] += 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  }
  __shared__ double sh[kRedThreads / 32][5];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < 5; ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) sh[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += sh[w][threadIdx.x];
    partials[blockIdx.x * 5 + threadIdx.x] = s;
  }
}

// Sum nblocks partial rows into out[5] (one block, fixed order).
__global__ void k_reduce_final(const double* partials, int nblocks, double* out);

// Boundary links of the fluid cell (x, y, z): bit q is set when its source
// x - c_q is not fluid (outside a non-periodic axis, or a non-zero flag),
// MASK_SPECIAL when one of those links is an INLET or OUTLET link; types
// receives the OR of those links' types.  The link-mask builder and the
// allocation-free reduction both take a cell's links from here.
template <class L>
__device__ __forceinline__ uint32_t cell_links(const Geom& g, const uint8_t* flags, int x, int y, int z,
                                               unsigned& types) {
  uint32_t m = 0;
  types = 0;
  for (int q = 1; q < L::Q; ++q) {
    int sx = x - L::cx(q), sy = y - L::cy(q), sz = z - L::cz(q);
    bool solid = false;
    if (sx < 0 || sx >= g.nx) { if (!g.per[0]) solid = true; else sx = (sx + g.nx) % g.nx; }
    if (sy < 0 || sy >= g.ny) { if (!g.per[1]) solid = true; else sy = (sy + g.ny) % g.ny; }
    if (sz < 0 || sz >= g.nz) { if (!g.per[2]) solid = true; else sz = (sz + g.nz) % g.nz; }
    int type = L_NOSLIP;
    if (!solid && flags != nullptr) {
      const uint8_t f = flags[sx + g.nx * (sy + g.ny * sz)];
      solid = !flag_is_fluid_source(f);
      if (solid) type = link_type_of_flag(f);
    }
    if (solid) {
      m |= 1u << q;
      if (type != L_NOSLIP) {
        m |= MASK_SPECIAL;
        types |= unsigned(type);
      }
    }
  }
  return m;
}

// Also ORs the types of all boundary links into *types (may be null).
template <class L>
__global__ void k_link_mask(const SweepArgs a, uint32_t* __restrict__ mask, unsigned* types) {
  const long long N = a.g.N;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    if (a.flags != nullptr && a.flags[cell] != 0) {
      mask[cell] = MASK_SOLID | (flag_is_ghost(a.flags[cell]) ? MASK_GHOST : 0u);
      continue;
    }
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    if (types != nullptr && ((!a.g.per[0] && x == a.g.nx - 1) || (!a.g.per[1] && y == a.g.ny - 1) ||
                             (!a.g.per[2] && z == a.g.nz - 1)))
      atomicOr(types, TYPES_FLUID_LAST_LAYER);
    if (types != nullptr && ((!a.g.per[0] && x == 0) || (!a.g.per[1] && y == 0) || (!a.g.per[2] && z == 0)))
      atomicOr(types, TYPES_FLUID_FIRST_LAYER);
    unsigned t = 0;
    mask[cell] = cell_links<L>(a.g, a.flags, x, y, z, t);
    if (types != nullptr && t != 0) atomicOr(types, t);
  }
}

// Initialisation by push: every cell forms its own P(x) (from FP64 rho/u or
// an FP64 P array) once and writes it where the layout needs it.  Pull
// layout: P_q(x) into slot q of its own cell.  AA natural layout (even
// parity): f_q(y) = P_q(y - c_q), so cell x pushes P_q(x) into slot q of
// y = x + c_q, exactly like the stores of the odd step; when y is not fluid
// the boundary value B_qbar(P(x)) goes to slot qbar of x instead.  Each slot
// is written once; non-fluid cells write their own slots.  Esoteric-twist
// layout (even parity): the writes of an odd esoteric-twist step; non-fluid
// cells write nothing.
template <class L, class ST, bool BND>
__global__ void __launch_bounds__(kBlockX) k_init_push(const SweepArgs a, int layout, int src_kind, const double* P,
                                                       const double* rho, const double* u) {
  using T = typename ST::T;
  using S = typename ST::S;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int cell = x + a.g.nx * (y + a.g.ny * z);
  const long long N = a.g.N;
  uint32_t mask = 0;
  if constexpr (BND) mask = a.mask[cell];
  // ghost cells receive their populations from the neighbouring block
  if (mask & MASK_GHOST) return;
  T v[L::Q];  // shifted populations h = P - w
  if (src_kind == 0) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) v[q] = T(P[q * N + cell] - L::w(q));
  } else {
    const T dr = T(rho[cell] - 1.0);
    const T r0 = a.cp.incompressible ? T(1) : T(1) + dr;
    const T uu[3] = {T(u[cell]), T(u[N + cell]), L::D == 3 ? T(u[2 * N + cell]) : T(0)};
    const T usq = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      const T cu = cdot<L, T>(q, uu);
      v[q] = T(L::w(q)) * (dr + r0 * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
    }
  }
  // esoteric twist: a solid cell's locations hold slots of its fluid
  // neighbours, so it writes nothing
  if (layout == 2 && (mask & MASK_SOLID)) return;
  if (layout == 0 || (mask & MASK_SOLID)) {
#pragma unroll
    for (int q = 0; q < L::Q; ++q) pdf_st<S>(a, a.dstq[q], cell, ST::from_h(v[q], L::w(q)));
    return;
  }
  if constexpr (BND) {
    if (mask & MASK_SPECIAL) {
      const OutletP op = outlet_params(a.cp);
      T up[3];
      post_velocity<L, T, true>(v, op, up);
      for (int q = 1; q < L::Q; ++q) {
        const int p = opp(q);
        if ((mask >> p) & 1u) {
          const int t = LBM_LINK_TYPE(a, x + L::cx(q), y + L::cy(q), z + L::cz(q));
          if (t == L_INLET) v[q] += ubb_term<L, T>(p, a.cp);
          else if (t == L_OUTLET) v[q] = outlet_value<L, T, true>(p, up, op);
        }
      }
    }
  }
  const Nbr nb = make_nbr(a.g, x, y, z);
  if (layout == 2) {
    // the writes of an odd esoteric-twist step: slot q at x + max(c_q, 0)
#pragma unroll
    for (int q = 0; q < L::Q; ++q) {
      const int p = opp(q);
      const bool b = BND && ((mask >> p) & 1u);
      const int idx = nb.at(eso_wr(L::cx(q)), eso_wr(L::cy(q)), eso_wr(L::cz(q)));
      pdf_st<S>(a, a.dstq[b ? p : q], idx, ST::from_h(v[q], L::w(q)));
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < L::Q; ++q) {
    const int p = opp(q);
    const bool b = BND && ((mask >> p) & 1u);
    const int qd = b ? p : q;
    const int idx = b ? cell : nb.at(L::cx(q), L::cy(q), L::cz(q));
    pdf_st<S>(a, a.dstq[qd], idx, ST::from_h(v[q], L::w(q)));
  }
}

// ------------------------------------------------------------ block halos
// x-slab blocks with one ghost layer on each x face (local x = 0 and nx - 1,
// cells flagged LBM_GHOST where the neighbouring block's cell is fluid).  The
// populations that cross a face between two steps depend on the pattern and
// the parity (Sec. IV-D: the single-array patterns are why the pack and
// unpack kernels are generated there).  For the face x = nx - 1 (side 1) and
// the directions q with c_x = +1 that cross it:
//   pack (what this block sends):
//     pull:            P_q at the last interior layer (x = nx - 2), slot q
//     AA, odd t:       the even step left P_q(x) in slot qbar of x = nx - 2
//     AA, even t > 0 or after initialisation: the odd step (or the push
//                      initialisation) wrote P_q of the last layer into slot
//                      q of the ghost layer x = nx - 1
//   unpack (what the neighbour across the face x = 0 stores):
//     pull: slot q of its ghost layer x = 0; AA odd t: slot qbar of x = 0;
//     AA even t: slot q of its first interior layer x = 1, except where that
//     slot holds the receiver's own boundary value (the link (x, q) comes
//     from a non-fluid cell across the face) or the cell is not fluid.
// The face x = 0 (side 0) mirrors this with the directions c_x = -1 and the
// layers 1, 0 (pack) and nx - 1, nx - 2 (unpack).  Buffer layout
// [k][z][y] for the k-th crossing direction, in the storage type.  Values
// for non-fluid positions travel too; they land in slots no sweep reads.
struct HaloSpec {
  int side;    // 0: face x = 0, 1: face x = nx - 1
  int mode;    // 0: pull, 1: AA with odd t, 2: AA with even t
  int unpack;  // 0: pack into buf, 1: unpack from buf
};

template <class L>
__host__ __device__ constexpr int halo_dirs() {
  int n = 0;
  for (int q = 0; q < L::Q; ++q) n += L::cx(q) == 1 ? 1 : 0;
  return n;
}

template <class L>
__device__ __forceinline__ int halo_dir(int k, int sign) {
  int n = 0;
  for (int q = 0; q < L::Q; ++q)
    if (L::cx(q) == sign) {
      if (n == k) return q;
      ++n;
    }
  return 0;
}

template <class L, class ST>
__global__ void k_halo(const SweepArgs a, HaloSpec h, typename ST::S* buf) {
  using S = typename ST::S;
  const long long plane = (long long)a.g.ny * a.g.nz;
  const long long total = plane * halo_dirs<L>();
  const int nx = a.g.nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = int(i / plane);
    const long long yz = i - k * plane;  // y + ny z
    // directions that cross the face outward (pack) or inward (unpack)
    const int sign = (h.side == 1) != (h.unpack != 0) ? 1 : -1;
    const int q = halo_dir<L>(k, sign);
    int x, slot;
    if (h.unpack == 0) {
      if (h.mode == 2) x = h.side == 1 ? nx - 1 : 0;
      else x = h.side == 1 ? nx - 2 : 1;
    } else {
      if (h.mode == 2) x = h.side == 1 ? nx - 2 : 1;
      else x = h.side == 1 ? nx - 1 : 0;
    }
    slot = h.mode == 1 ? opp(q) : q;
    const long long cell = x + (long long)nx * yz;
    S* p = static_cast<S*>(a.dst) + (long long)slot * a.g.N + cell;
    if (h.unpack == 0) {
      buf[i] = *p;
    } else {
      // into an interior cell (AA, even t): not where the receiver keeps a
      // boundary value of its own (a non-fluid cell, or a link whose source
      // across the face is non-fluid, whose slot the receiver's odd step
      // filled with B_q)
      if (h.mode == 2 && a.mask != nullptr) {
        const uint32_t m = a.mask[cell];
        if ((m & MASK_SOLID) || ((m >> q) & 1u)) continue;
      }
      *p = buf[i];
    }
  }
}

// --------------------------------------------------------------- launchers
// A stream beside the sweep's own for the second launch of a list sweep
// (the cells on a face of a periodic axis, and for the two-grid pull the
// cells with inlet or outlet links).  Within one step every cell reads and
// writes only slots no other cell touches (pull: its own destination
// slots; AA and the esoteric twist: the slots of its own links), so the two
// launches can run at once: the second is forked off the sweep's stream
// before the main launch and joined back after it, and the next step waits
// for both.  Null: both launches run in order on the sweep's stream.
struct SideStream {
  cudaStream_t s;
  cudaEvent_t fork, join;
};

inline dim3 sweep_block(const Geom& g) {
  int bx = g.nx >= kBlockX ? kBlockX : ((g.nx + 31) / 32) * 32;
  return dim3(bx, 1, 1);
}
inline dim3 sweep_grid(const Geom& g) {
  const dim3 b = sweep_block(g);
  return dim3((g.nx + b.x - 1) / b.x, g.ny, g.nz);
}
// blocks of a sweep_grid launch (rows of the adjoint's force scratch)
inline long long adjoint_rows(const Geom& g) {
  const dim3 gr = sweep_grid(g);
  return (long long)gr.x * gr.y * gr.z;
}

template <class L, class ST, int OP, int KIND>
cudaError_t launch_sweep_k(bool bnd, const SweepArgs& a, cudaStream_t s, const SideStream* side) {
  if constexpr (ST::ID == StF16S::ID) {
    if (!bnd && (a.g.nx % 2) == 0) {
      Geom half = a.g;
      half.nx = a.g.nx / 2;
      SweepArgs b = a;
      if constexpr (KIND == K_AA_EVEN) {
        // population prefetch distance: a third of the cells resident at once
        static long long resident_cells = 0;
        if (resident_cells == 0) {
          int dev = 0, sms = 0, per_sm = 0;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_h2<L, OP, KIND>, kBlockX, 0);
          resident_cells = 2LL * (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) * kBlockX;
        }
        b.pop_ahead = int(resident_cells / 3) & ~(2 * kBlockX - 1);  // whole blocks of cell pairs
      }
      k_sweep_h2<L, OP, KIND><<<sweep_grid(half), sweep_block(half), 0, s>>>(b);
      return cudaGetLastError();
    }
  }
  if (!bnd) {
    if constexpr (light_op<ST, OP>())
      k_sweep_light<L, ST, OP, KIND><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a);
    else
      k_sweep<L, ST, OP, KIND><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a);
    return cudaGetLastError();
  }
  const bool fork = side != nullptr && a.n_main > 0 && a.n_wrap > 0;
  if (fork) {
    cudaError_t e = cudaEventRecord(side->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side->s, side->fork, 0);
    if (e != cudaSuccess) return e;
    k_sweep_list_wrap<L, ST, OP, KIND><<<(a.n_wrap + kBlockX - 1) / kBlockX, kBlockX, 0, side->s>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(side->join, side->s);
    if (e != cudaSuccess) return e;
  }
  if (a.n_main > 0) {
    // entry prefetch distance: one and a half times the threads resident at
    // once (blocks per SM from the occupancy calculator, per instantiation)
    static int resident = 0;
    if (resident == 0) {
      int dev = 0, sms = 0, per_sm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if constexpr (list_capped<L, ST, OP>())
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_list_capped<L, ST, OP, KIND>, kBlockX, 0);
      else if constexpr (light_op<ST, OP>())
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_list_light<L, ST, OP, KIND>, kBlockX, 0);
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_list<L, ST, OP, KIND>, kBlockX, 0);
      resident = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) * kBlockX;
    }
    SweepArgs b = a;
    b.list_ahead = resident + resident / 2;
    b.pop_ahead = (KIND == K_AA_EVEN || KIND == K_AA_ODD) ? resident / 3 : 0;
    const int nb = (a.n_main + kBlockX - 1) / kBlockX;
    if constexpr (list_capped<L, ST, OP>())
      k_sweep_list_capped<L, ST, OP, KIND><<<nb, kBlockX, 0, s>>>(b);
    else if constexpr (light_op<ST, OP>())
      k_sweep_list_light<L, ST, OP, KIND><<<nb, kBlockX, 0, s>>>(b);
    else
      k_sweep_list<L, ST, OP, KIND><<<nb, kBlockX, 0, s>>>(b);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fork) return cudaStreamWaitEvent(s, side->join, 0);
  if (a.n_wrap > 0) k_sweep_list_wrap<L, ST, OP, KIND><<<(a.n_wrap + kBlockX - 1) / kBlockX, kBlockX, 0, s>>>(a);
  return cudaGetLastError();
}

template <class L, class ST, int OP>
cudaError_t launch_sweep_op(int kind, bool bnd, const SweepArgs& a, cudaStream_t s, const SideStream* side) {
  switch (kind) {
    case K_PULL: return launch_sweep_k<L, ST, OP, K_PULL>(bnd, a, s, side);
    case K_AA_EVEN: return launch_sweep_k<L, ST, OP, K_AA_EVEN>(bnd, a, s, side);
    case K_AA_ODD: return launch_sweep_k<L, ST, OP, K_AA_ODD>(bnd, a, s, side);
    case K_ESO_EVEN: return launch_sweep_k<L, ST, OP, K_ESO_EVEN>(bnd, a, s, side);
    case K_ESO_ODD: return launch_sweep_k<L, ST, OP, K_ESO_ODD>(bnd, a, s, side);
  }
  return cudaErrorInvalidValue;
}

inline int grid_stride_blocks(long long N, int threads) {
  long long b = (N + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace lbm
