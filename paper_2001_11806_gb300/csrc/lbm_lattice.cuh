// Lattice velocity sets, weights and storage conversions for the CUDA path.
//
// DdQq stencils (Sec. III-A): integer velocities in {-1,0,1}^d, c_s^2 = 1/3.
// D2Q9 and D3Q27 weights are products of the 1-D weights {2/3, 1/6, 1/6};
// D3Q19 uses the standard Hermite weights 1/3, 1/18, 1/36.  The direction
// order is the one documented in include/lbm.h (rest, faces, edges, corners;
// opposite directions adjacent, odd index q paired with q + 1).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

// Velocity table for the 27 velocities of D3Q27 in ABI order; D2Q9 and
// D3Q19 use prefixes/subsets of it (see the stencil structs).
struct Vel { int x, y, z; };

__host__ __device__ constexpr Vel vel27(int q) {
  constexpr Vel t[27] = {
      {0, 0, 0},
      {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
      {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
      {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
      {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
      {1, 1, 1},  {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
      {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
  return t[q];
}

__host__ __device__ constexpr Vel vel9(int q) {
  constexpr Vel t[9] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
  return t[q];
}

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

struct D2Q9 {
  static constexpr int Q = 9, D = 2, ID = 0;
  __host__ __device__ static constexpr int cx(int q) { return vel9(q).x; }
  __host__ __device__ static constexpr int cy(int q) { return vel9(q).y; }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int q) { return w1d(cx(q)) * w1d(cy(q)); }
  // weight numerator over 36 = 6^2: a factor 4 per zero component
  __host__ __device__ static constexpr long long w_num(int q) { return (cx(q) == 0 ? 4 : 1) * (cy(q) == 0 ? 4 : 1); }
  static constexpr long long w_den = 36;
};

struct D3Q19 {
  static constexpr int Q = 19, D = 3, ID = 1;
  __host__ __device__ static constexpr int cx(int q) { return vel27(q).x; }
  __host__ __device__ static constexpr int cy(int q) { return vel27(q).y; }
  __host__ __device__ static constexpr int cz(int q) { return vel27(q).z; }
  __host__ __device__ static constexpr int c2(int q) { return cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q); }
  __host__ __device__ static constexpr double w(int q) {
    return c2(q) == 0 ? 1.0 / 3.0 : (c2(q) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr long long w_num(int q) { return c2(q) == 0 ? 12 : (c2(q) == 1 ? 2 : 1); }
  static constexpr long long w_den = 36;
};

struct D3Q27 {
  static constexpr int Q = 27, D = 3, ID = 2;
  __host__ __device__ static constexpr int cx(int q) { return vel27(q).x; }
  __host__ __device__ static constexpr int cy(int q) { return vel27(q).y; }
  __host__ __device__ static constexpr int cz(int q) { return vel27(q).z; }
  __host__ __device__ static constexpr double w(int q) { return w1d(cx(q)) * w1d(cy(q)) * w1d(cz(q)); }
  __host__ __device__ static constexpr long long w_num(int q) {
    return (cx(q) == 0 ? 4 : 1) * (cy(q) == 0 ? 4 : 1) * (cz(q) == 0 ? 4 : 1);
  }
  static constexpr long long w_den = 216;
};

__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

// ------------------------------------------------------------- storage types
// Each storage trait converts between the stored value and the shifted
// population h = f - w_q used in registers (T is the compute type).
struct StF64 {
  using S = double; using T = double;
  static constexpr int ID = 0; static constexpr bool shifted = false;
  __device__ static __forceinline__ T to_h(S s, double w) { return s - w; }
  __device__ static __forceinline__ S from_h(T h, double w) { return h + w; }
  __device__ static __forceinline__ double to_f64(S s, double w) { return s; }
  __device__ static __forceinline__ S from_f64(double f, double w) { return f; }
};
struct StF32 {
  using S = float; using T = float;
  static constexpr int ID = 1; static constexpr bool shifted = false;
  __device__ static __forceinline__ T to_h(S s, double w) { return s - (float)w; }
  __device__ static __forceinline__ S from_h(T h, double w) { return h + (float)w; }
  __device__ static __forceinline__ double to_f64(S s, double w) { return (double)s; }
  __device__ static __forceinline__ S from_f64(double f, double w) { return (float)f; }
};
struct StF16S {
  using S = __half; using T = float;
  static constexpr int ID = 2; static constexpr bool shifted = true;
  __device__ static __forceinline__ T to_h(S s, double) { return __half2float(s); }
  __device__ static __forceinline__ S from_h(T h, double) { return __float2half_rn(h); }
  __device__ static __forceinline__ double to_f64(S s, double w) { return (double)__half2float(s) + w; }
  __device__ static __forceinline__ S from_f64(double f, double w) { return __double2half(f - w); }
};
struct StF32S {
  using S = float; using T = float;
  static constexpr int ID = 3; static constexpr bool shifted = true;
  __device__ static __forceinline__ T to_h(S s, double) { return s; }
  __device__ static __forceinline__ S from_h(T h, double) { return h; }
  __device__ static __forceinline__ double to_f64(S s, double w) { return (double)s + w; }
  __device__ static __forceinline__ S from_f64(double f, double w) { return (float)(f - w); }
};

// Flag bits (uint8 per cell) and link-mask bits, as in include/lbm.h.
enum : uint8_t { F_NOSLIP = 1, F_INLET = 2, F_OUTLET = 4, F_GHOST = 8 };
constexpr uint32_t MASK_SOLID = 0x80000000u;
constexpr uint32_t MASK_SPECIAL = 0x40000000u;  // the cell has an inlet or outlet link
constexpr uint32_t MASK_GHOST = 0x20000000u;    // a ghost cell (also MASK_SOLID: not swept)

// A ghost cell (GHOST bit without NOSLIP, INLET or OUTLET) holds populations
// of a neighbouring block: it is not swept, but links from it stream like
// fluid links.
__host__ __device__ inline bool flag_is_ghost(uint8_t f) { return (f & 7) == 0 && (f & F_GHOST) != 0; }
__host__ __device__ inline bool flag_is_fluid_source(uint8_t f) { return f == 0 || flag_is_ghost(f); }
enum LinkType : int { L_NOSLIP = 1, L_INLET = 2, L_OUTLET = 4 };

__host__ __device__ inline int link_type_of_flag(uint8_t f) {
  if (f & F_NOSLIP) return L_NOSLIP;
  if (f & F_INLET) return L_INLET;
  if (f & F_OUTLET) return L_OUTLET;
  return L_NOSLIP;
}

}  // namespace lbm
