// Dispatch tables: everything that depends on (stencil, storage) is
// reached through one OpsTable per pair, built in lbm_inst_*.cu.
#pragma once
#include "lbm_adjoint.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

// Everything that depends on (stencil, storage): explicitly instantiated in
// one translation unit per pair.
template <class L, class ST>
struct Ops {
  static cudaError_t sweep(int op, int kind, bool bnd, const SweepArgs& a, cudaStream_t s, const SideStream* side) {
    switch (op) {
      case OP_SRT: return launch_sweep_op<L, ST, OP_SRT>(kind, bnd, a, s, side);
      case OP_TRT: return launch_sweep_op<L, ST, OP_TRT>(kind, bnd, a, s, side);
      case OP_MRT: return launch_sweep_op<L, ST, OP_MRT>(kind, bnd, a, s, side);
      case OP_SRT_LES: return launch_sweep_op<L, ST, OP_SRT_LES>(kind, bnd, a, s, side);
      case OP_TRT_LES: return launch_sweep_op<L, ST, OP_TRT_LES>(kind, bnd, a, s, side);
      case OP_KBC: return launch_sweep_op<L, ST, OP_KBC>(kind, bnd, a, s, side);
      case OP_MRT3: return launch_sweep_op<L, ST, OP_MRT3>(kind, bnd, a, s, side);
      case OP_CUM:
        if constexpr (L::Q == 27) return launch_sweep_op<L, ST, OP_CUM>(kind, bnd, a, s, side);
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t populations(int view, const SweepArgs& a, double* out, cudaStream_t s) {
    k_populations<L, ST><<<grid_stride_blocks(a.g.N, 256), 256, 0, s>>>(a, view, out);
    return cudaGetLastError();
  }
  static cudaError_t macroscopic(int view, const SweepArgs& a, void* rho, void* u, bool f64, cudaStream_t s) {
    if (f64)
      k_macroscopic<L, ST, double><<<grid_stride_blocks(a.g.N, 256), 256, 0, s>>>(a, view, (double*)rho, (double*)u);
    else
      k_macroscopic<L, ST, float><<<grid_stride_blocks(a.g.N, 256), 256, 0, s>>>(a, view, (float*)rho, (float*)u);
    return cudaGetLastError();
  }
  static cudaError_t reduce_partial(int view, const SweepArgs& a, double* partials, int nblocks, cudaStream_t s) {
    k_reduce_partial<L, ST><<<nblocks, kRedThreads, 0, s>>>(a, view, partials);
    return cudaGetLastError();
  }
  // layout: 0 two-grid (P in place), 1 AA natural, 2 esoteric twist even
  static cudaError_t set_state(int layout, int src_kind, const SweepArgs& a, const double* P, const double* rho,
                               const double* u, cudaStream_t s) {
    if (a.mask != nullptr)
      k_init_push<L, ST, true><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a, layout, src_kind, P, rho, u);
    else
      k_init_push<L, ST, false><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a, layout, src_kind, P, rho, u);
    return cudaGetLastError();
  }
  using T = typename ST::T;
  // rows: scratch of adjoint_rows(g) x 3 doubles for the per-block force
  // sums when dF is non-null (and the sweep has a force)
  template <int OP>
  static cudaError_t adjoint_op(bool bnd, const SweepArgs& a, const void* li, void* lo, double* dF, double* rows,
                                cudaStream_t s) {
    double* r = (dF != nullptr && a.cp.has_force) ? rows : nullptr;
    if (bnd)
      k_adjoint<L, ST, OP, true><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a, (const T*)li, (T*)lo, r);
    else
      k_adjoint<L, ST, OP, false><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a, (const T*)li, (T*)lo, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || r == nullptr) return e;
    k_force_rows_final<double><<<1, kForceThreads, 0, s>>>(r, adjoint_rows(a.g), dF);
    return cudaGetLastError();
  }
  static cudaError_t adjoint(int op, bool bnd, const SweepArgs& a, const void* li, void* lo, double* dF,
                             double* rows, cudaStream_t s) {
    switch (op) {
      case OP_SRT: return adjoint_op<OP_SRT>(bnd, a, li, lo, dF, rows, s);
      case OP_TRT: return adjoint_op<OP_TRT>(bnd, a, li, lo, dF, rows, s);
      case OP_MRT: return adjoint_op<OP_MRT>(bnd, a, li, lo, dF, rows, s);
    }
    return cudaErrorInvalidValue;
  }
  static cudaError_t ke_seed(bool bnd, const SweepArgs& a, const int* box, double* loss, void* lo, double* dF,
                             cudaStream_t s) {
    const int4 lo4 = make_int4(box[0], box[2], box[4], 0), hi4 = make_int4(box[1], box[3], box[5], 0);
    if (bnd)
      k_ke_seed<L, ST, true><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a, lo4, hi4, loss, (T*)lo, dF);
    else
      k_ke_seed<L, ST, false><<<sweep_grid(a.g), sweep_block(a.g), 0, s>>>(a, lo4, hi4, loss, (T*)lo, dF);
    return cudaGetLastError();
  }
  static cudaError_t eq_vjp(const SweepArgs& a, const double* rho0, const double* u0, const void* lam, double* g,
                            cudaStream_t s) {
    k_eq_vjp<L, T><<<grid_stride_blocks(a.g.N, 256), 256, 0, s>>>(a, rho0, u0, (const T*)lam, g);
    return cudaGetLastError();
  }
};

template <class L, class ST>
cudaError_t launch_halo(const SweepArgs& a, HaloSpec h, void* buf, cudaStream_t s) {
  const long long n = (long long)a.g.ny * a.g.nz * halo_dirs<L>();
  k_halo<L, ST><<<grid_stride_blocks(n, 256), 256, 0, s>>>(a, h, static_cast<typename ST::S*>(buf));
  return cudaGetLastError();
}

template <class L>
cudaError_t launch_link_mask(const SweepArgs& a, uint32_t* mask, unsigned* types, cudaStream_t s) {
  k_link_mask<L><<<grid_stride_blocks(a.g.N, 256), 256, 0, s>>>(a, mask, types);
  return cudaGetLastError();
}

template <class L, class ST>
cudaError_t launch_boundary_pull(const SweepArgs& a, void* P, cudaStream_t s) {
  const int n = a.n_main + a.n_wrap;
  if (n > 0)
    k_boundary_pull<L, ST><<<(n + kBlockX - 1) / kBlockX, kBlockX, 0, s>>>(a, static_cast<typename ST::S*>(P));
  return cudaGetLastError();
}

template <class L>
cudaError_t launch_list_count(const SweepArgs& a, int nblk, int* counts, cudaStream_t s) {
  k_list_count<L><<<nblk, kListThreads, 0, s>>>(a, nblk, counts);
  return cudaGetLastError();
}

template <class L>
cudaError_t launch_list_scatter(const SweepArgs& a, int nblk, const int* offsets, uint2* list, cudaStream_t s) {
  k_list_scatter<L><<<nblk, kListThreads, 0, s>>>(a, nblk, offsets, list);
  return cudaGetLastError();
}

// Dispatch table of one (stencil, storage) pair.  Each lbm_inst_*.cu defines
// one factory returning it, so the C ABI unit instantiates no kernels.
struct OpsTable {
  cudaError_t (*sweep)(int, int, bool, const SweepArgs&, cudaStream_t, const SideStream*);
  cudaError_t (*populations)(int, const SweepArgs&, double*, cudaStream_t);
  cudaError_t (*macroscopic)(int, const SweepArgs&, void*, void*, bool, cudaStream_t);
  cudaError_t (*reduce_partial)(int, const SweepArgs&, double*, int, cudaStream_t);
  cudaError_t (*set_state)(int, int, const SweepArgs&, const double*, const double*, const double*, cudaStream_t);
  cudaError_t (*link_mask)(const SweepArgs&, uint32_t*, unsigned*, cudaStream_t);
  cudaError_t (*adjoint)(int, bool, const SweepArgs&, const void*, void*, double*, double*, cudaStream_t);
  cudaError_t (*ke_seed)(bool, const SweepArgs&, const int*, double*, void*, double*, cudaStream_t);
  cudaError_t (*eq_vjp)(const SweepArgs&, const double*, const double*, const void*, double*, cudaStream_t);
  cudaError_t (*list_count)(const SweepArgs&, int, int*, cudaStream_t);
  cudaError_t (*list_scatter)(const SweepArgs&, int, const int*, uint2*, cudaStream_t);
  cudaError_t (*boundary_pull)(const SweepArgs&, void*, cudaStream_t);
  cudaError_t (*halo)(const SweepArgs&, HaloSpec, void*, cudaStream_t);
};

template <class L, class ST>
OpsTable make_table() {
  return OpsTable{&Ops<L, ST>::sweep,          &Ops<L, ST>::populations, &Ops<L, ST>::macroscopic,
                  &Ops<L, ST>::reduce_partial, &Ops<L, ST>::set_state,   &launch_link_mask<L>,
                  &Ops<L, ST>::adjoint,        &Ops<L, ST>::ke_seed,     &Ops<L, ST>::eq_vjp,
                  &launch_list_count<L>,       &launch_list_scatter<L>,  &launch_boundary_pull<L, ST>,
                  &launch_halo<L, ST>};
}

#define LBM_TABLE_DECL(l, s) OpsTable ops_table_##l##_##s();
#define LBM_ALL_TABLES(X) \
  X(d2q9, f64) X(d2q9, f32) X(d2q9, f16s) X(d2q9, f32s) \
  X(d3q19, f64) X(d3q19, f32) X(d3q19, f16s) X(d3q19, f32s) \
  X(d3q27, f64) X(d3q27, f32) X(d3q27, f16s) X(d3q27, f32s)
LBM_ALL_TABLES(LBM_TABLE_DECL)


}  // namespace lbm
