// C ABI of liblbm.so (declared in include/lbm.h): validation, buffer
// bookkeeping and dispatch to the kernels instantiated per stencil/storage.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/lbm.h"
#include "lbm_ops.cuh"

namespace lbm {
__global__ void k_reduce_final(const double* partials, int nblocks, double* out) {
  if (threadIdx.x < 5) {
    double s = 0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

OpsTable get_table(int stencil, int storage) {
  switch (stencil * 4 + storage) {
    case LBM_D2Q9 * 4 + LBM_F64: return ops_table_d2q9_f64();
    case LBM_D2Q9 * 4 + LBM_F32: return ops_table_d2q9_f32();
    case LBM_D2Q9 * 4 + LBM_F16S: return ops_table_d2q9_f16s();
    case LBM_D2Q9 * 4 + LBM_F32S: return ops_table_d2q9_f32s();
    case LBM_D3Q19 * 4 + LBM_F64: return ops_table_d3q19_f64();
    case LBM_D3Q19 * 4 + LBM_F32: return ops_table_d3q19_f32();
    case LBM_D3Q19 * 4 + LBM_F16S: return ops_table_d3q19_f16s();
    case LBM_D3Q19 * 4 + LBM_F32S: return ops_table_d3q19_f32s();
    case LBM_D3Q27 * 4 + LBM_F64: return ops_table_d3q27_f64();
    case LBM_D3Q27 * 4 + LBM_F32: return ops_table_d3q27_f32();
    case LBM_D3Q27 * 4 + LBM_F16S: return ops_table_d3q27_f16s();
    default: return ops_table_d3q27_f32s();
  }
}

template <class L>
void mrt_factors(const double* omega, CollideParams& cp) {
  constexpr auto& B = mrt::Table<L>::B;
  for (int k = 0; k < 27; ++k) { cp.mrt_s[k] = 0.f; cp.mrt_s_d[k] = 0.0; }
  for (int k = 0; k < L::Q; ++k) {
    const double s = B.group[k] < 0 ? 0.0 : omega[B.group[k]];
    cp.mrt_s_d[k] = s * B.invD[k];
    cp.mrt_s[k] = (float)cp.mrt_s_d[k];
  }
}

}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
  lbm_params p;
  int q = 0, d = 0;
  long long N = 0;
  size_t elem = 0, pdf_bytes = 0, aux_bytes = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;  // pull: index of the buffer that holds P
  void* aux = nullptr;
  const uint8_t* flags = nullptr;
  uint32_t* mask = nullptr;
  double* partials = nullptr;
  double* force_rows = nullptr;  // per-block body-force sums of the adjoint sweep
  double* result = nullptr;
  bool has_mask = false;
  uint2* list = nullptr;  // fluid cells of a masked domain with their mask words (SweepArgs::list)
  int n_main = 0, n_wrap = 0;
  unsigned link_types = 0;  // OR of the boundary-link types present (L_INLET, L_OUTLET)
  cudaStream_t stream = nullptr;
  int64_t t = 0;
  int kernel_op = 0;  // collision operator of the sweep kernels (LES variants included)
  CollideParams cp;
  OpsTable ops;
  char err[256] = {0};  // last error text; fixed storage, so reporting never allocates
  // Small domains: lbm_step replays kGraphSteps sweeps as one CUDA graph
  // (recorded on a private stream; index = pull buffer holding P, 0 for the
  // single-array patterns, which start a graph at even parity).
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // list sweeps with a second launch: the stream and events that run it
  // beside the main launch (SideStream; s null when the list has no second
  // part)
  SideStream side = {nullptr, nullptr, nullptr};
  const SideStream* side_or_null() const { return side.s ? &side : nullptr; }
  ~lbm_ctx() {
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side.join) cudaEventDestroy(side.join);
    if (side.fork) cudaEventDestroy(side.fork);
    if (side.s) cudaStreamDestroy(side.s);
  }
};

namespace {

const char* kStatusNames[] = {"LBM_OK", "LBM_E_INVAL", "LBM_E_UNSUPPORTED", "LBM_E_CUDA", "LBM_E_NOMEM",
                              "LBM_E_BUFSIZE", "LBM_E_NONFINITE", "LBM_E_BOUNDS", "LBM_E_STATE"};

// CUDA graphs for small domains, where a sweep is shorter than its launch.
constexpr int kGraphSteps = 32;
constexpr long long kGraphMaxCells = 1 << 20;

struct Layout {
  size_t mask_off, mask_bytes, list_off, count_off, part_off, adj_off, res_off, total;
  int nblk;  // chunks of the fluid-list builder
};

int stencil_q(int s) { return s == LBM_D2Q9 ? 9 : (s == LBM_D3Q19 ? 19 : 27); }
int stencil_d(int s) { return s == LBM_D2Q9 ? 2 : 3; }
size_t storage_bytes(int st) { return st == LBM_F64 ? 8 : (st == LBM_F16S ? 2 : 4); }
size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool needs_mask(const lbm_params& p, bool has_flags) {
  if (has_flags) return true;
  const int d = stencil_d(p.stencil);
  for (int a = 0; a < d; ++a)
    if (!p.periodic[a]) return true;
  return false;
}

// aux = [link mask: 4 N bytes][fluid-cell list: 8 N bytes][list-builder
// counts: 2 x 4 x nblk bytes][reduction partials][adjoint force rows: 3
// doubles per sweep block][reduction result]; the mask
// and list regions are always reserved so that the size does not depend on
// the flags.
Layout layout_for(const lbm_params& p, long long N) {
  Layout l;
  l.nblk = int((N + kListChunk - 1) / kListChunk);
  l.mask_off = 0;
  l.mask_bytes = align256(size_t(N) * 4);
  l.list_off = l.mask_bytes;
  l.count_off = l.list_off + align256(size_t(N) * 8);
  l.part_off = l.count_off + align256(size_t(l.nblk) * 2 * sizeof(int));
  Geom g{};
  g.nx = p.nx;
  g.ny = p.ny;
  g.nz = p.nz;
  l.adj_off = l.part_off + align256(size_t(kRedMaxBlocks) * 5 * sizeof(double));
  l.res_off = l.adj_off + align256(size_t(adjoint_rows(g)) * 3 * sizeof(double));
  l.total = l.res_off + 256;
  return l;
}

bool rate_ok(double w) { return std::isfinite(w) && w > 0.0 && w < 2.0; }

// Validate parameters; fills msg on failure.
lbm_status validate(const lbm_params* p, const char** msg) {
  if (!p) { *msg = "params is NULL"; return LBM_E_INVAL; }
  if (p->stencil < LBM_D2Q9 || p->stencil > LBM_D3Q27) { *msg = "unknown stencil"; return LBM_E_INVAL; }
  if (p->collision < LBM_SRT || p->collision > LBM_KBC) { *msg = "unknown collision"; return LBM_E_INVAL; }
  if (p->storage < LBM_F64 || p->storage > LBM_F32S) { *msg = "unknown storage"; return LBM_E_INVAL; }
  if (p->pattern != LBM_PULL && p->pattern != LBM_AA && p->pattern != LBM_ESOTWIST) {
    *msg = "unknown pattern";
    return LBM_E_INVAL;
  }
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) { *msg = "nx, ny, nz must be >= 1"; return LBM_E_INVAL; }
  if (p->stencil == LBM_D2Q9 && p->nz != 1) { *msg = "D2Q9 needs nz == 1"; return LBM_E_INVAL; }
  if (p->ny > 65535 || p->nz > 65535) { *msg = "ny and nz must be <= 65535"; return LBM_E_INVAL; }
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > 2147483647LL) { *msg = "more than 2^31-1 cells"; return LBM_E_INVAL; }
  switch (p->collision) {
    case LBM_SRT:
      if (!rate_ok(p->omega[0])) { *msg = "omega[0] must be in (0, 2)"; return LBM_E_INVAL; }
      break;
    case LBM_TRT:
      if (!rate_ok(p->omega[0])) { *msg = "omega_e must be in (0, 2)"; return LBM_E_INVAL; }
      if (p->trt_magic) {
        if (!(p->magic > 0.0) || !std::isfinite(p->magic)) { *msg = "magic must be > 0"; return LBM_E_INVAL; }
      } else if (!rate_ok(p->omega[1])) {
        *msg = "omega_o must be in (0, 2)";
        return LBM_E_INVAL;
      }
      break;
    case LBM_MRT: {
      const int nr = p->stencil == LBM_D3Q27 ? 6 : 4;
      for (int i = 0; i < nr; ++i)
        if (!rate_ok(p->omega[i])) { *msg = "MRT rates must be in (0, 2)"; return LBM_E_INVAL; }
      break;
    }
    case LBM_CUMULANT:
      for (int i = 0; i < 3; ++i)
        if (!rate_ok(p->omega[i])) { *msg = "cumulant rates must be in (0, 2)"; return LBM_E_INVAL; }
      if (p->stencil != LBM_D3Q27) { *msg = "the cumulant operator is built for D3Q27 only"; return LBM_E_UNSUPPORTED; }
      if (p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0) {
        *msg = "cumulant collision with a body force is not built";
        return LBM_E_UNSUPPORTED;
      }
      if (p->incompressible) { *msg = "incompressible cumulant collision is not built"; return LBM_E_UNSUPPORTED; }
      break;
    case LBM_KBC:
      for (int i = 0; i < 2; ++i)
        if (!rate_ok(p->omega[i])) { *msg = "KBC shear and bulk rates must be in (0, 2)"; return LBM_E_INVAL; }
      if (p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0) {
        *msg = "KBC collision with a body force is not built";
        return LBM_E_UNSUPPORTED;
      }
      break;
  }
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(p->force[i]) || !std::isfinite(p->u_wall[i])) { *msg = "non-finite force or wall velocity"; return LBM_E_INVAL; }
  if (!(p->rho_outlet > 0.0) || !std::isfinite(p->rho_outlet)) { *msg = "rho_outlet must be > 0"; return LBM_E_INVAL; }
  if (!(p->smagorinsky_cs >= 0.0) || !std::isfinite(p->smagorinsky_cs)) {
    *msg = "smagorinsky_cs must be >= 0";
    return LBM_E_INVAL;
  }
  if (p->boundary_mode != LBM_BOUNDARY_IN_SWEEP && p->boundary_mode != LBM_BOUNDARY_SEPARATE) {
    *msg = "unknown boundary_mode";
    return LBM_E_INVAL;
  }
  if (p->boundary_mode == LBM_BOUNDARY_SEPARATE && p->pattern != LBM_PULL) {
    *msg = "separate boundary kernels are built for the two-grid pull pattern";
    return LBM_E_UNSUPPORTED;
  }
  if (p->smagorinsky_cs > 0.0 && p->collision != LBM_SRT && p->collision != LBM_TRT) {
    *msg = "the Smagorinsky model is built for SRT and TRT";
    return LBM_E_UNSUPPORTED;
  }
  return LBM_OK;
}

// Last-error text, truncated to the fixed buffer.
void set_err(lbm_ctx* c, const char* a, const char* b = "", const char* d = "") {
  std::snprintf(c->err, sizeof(c->err), "%s%s%s", a, b, d);
}

// Host allocations that lbm_debug_fail_host_allocs asked to fail.
std::atomic<int> g_fail_allocs{0};
bool injected_alloc_failure() {
  int n = g_fail_allocs.load();
  while (n > 0)
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
  return false;
}

// Fluid-cell list of a masked domain (see k_sweep_list): per-chunk counts on
// the device, exclusive offsets on the host, ordered scatter on the device.
lbm_status build_list(lbm_ctx* c, const SweepArgs& a, const Layout& lay) {
  int* counts = reinterpret_cast<int*>(static_cast<char*>(c->aux) + lay.count_off);
  const int nblk = lay.nblk;
  const size_t nh = size_t(nblk) * 2;
  int* h = injected_alloc_failure() ? nullptr : static_cast<int*>(std::malloc(nh * sizeof(int)));
  if (!h) {
    set_err(c, "host allocation of the list offsets failed");
    return LBM_E_NOMEM;
  }
  struct Free {
    int* p;
    ~Free() { std::free(p); }
  } guard{h};
  cudaError_t e = c->ops.list_count(a, nblk, counts, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, counts, nh * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    set_err(c, "list count: ", cudaGetErrorString(e));
    return LBM_E_CUDA;
  }
  long long n_main = 0;
  for (int b = 0; b < nblk; ++b) n_main += h[b];
  long long run1 = 0, run2 = n_main;
  for (int b = 0; b < nblk; ++b) {
    const int k1 = h[b], k2 = h[size_t(nblk) + b];
    h[b] = int(run1);
    h[size_t(nblk) + b] = int(run2);
    run1 += k1;
    run2 += k2;
  }
  c->n_main = int(n_main);
  c->n_wrap = int(run2 - n_main);
  e = cudaMemcpyAsync(counts, h, nh * sizeof(int), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = c->ops.list_scatter(a, nblk, counts, c->list, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    set_err(c, "list scatter: ", cudaGetErrorString(e));
    return LBM_E_CUDA;
  }
  return LBM_OK;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  set_err(c, where, ": ", cudaGetErrorString(e));
  return LBM_E_CUDA;
}

// Device word of the bounds-checking build (in the aux result area).
unsigned* bounds_word(const lbm_ctx* c) {
  return c->result ? reinterpret_cast<unsigned*>(reinterpret_cast<char*>(c->result) + 72) : nullptr;
}

// Bounds-checking build: waits for the stream and turns a recorded
// out-of-array access into LBM_E_BOUNDS (the word is cleared).  Otherwise a
// no-op.
lbm_status debug_check(lbm_ctx* c) {
#ifdef LBM_DEBUG_BOUNDS
  unsigned word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, bounds_word(c), sizeof(word), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return LBM_E_CUDA;
  if (word) {
    cudaMemsetAsync(bounds_word(c), 0, sizeof(unsigned), c->stream);
    std::snprintf(c->err, sizeof(c->err), "a kernel accessed memory outside the population arrays");
    return LBM_E_BOUNDS;
  }
#else
  (void)c;
#endif
  return LBM_OK;
}

SweepArgs make_args(const lbm_ctx* c, const void* src, void* dst) {
  SweepArgs a;
  a.src = src;
  a.dst = dst;
  a.mask = c->has_mask ? c->mask : nullptr;
  a.flags = c->flags;
  a.g.nx = c->p.nx;
  a.g.ny = c->p.ny;
  a.g.nz = c->p.nz;
  for (int i = 0; i < 3; ++i) a.g.per[i] = c->p.periodic[i] ? 1 : 0;
  if (c->d == 2) a.g.per[2] = 1;
  a.g.N = c->N;
  a.cp = c->cp;
  a.list = c->list;
  a.n_main = c->n_main;
  a.n_wrap = c->n_wrap;
  a.boundary_mode = c->p.boundary_mode;
  a.special_wrap = (c->p.pattern == LBM_PULL && c->p.boundary_mode == LBM_BOUNDARY_IN_SWEEP) ? 1 : 0;
  a.list_ahead = 0;
  a.pop_ahead = 0;
  a.pdf_bytes = c->pdf_bytes;
  a.bounds_flag = bounds_word(c);
  for (int q = 0; q < 27; ++q) {
    const size_t off = q < c->q ? size_t(q) * size_t(c->N) * c->elem : 0;
    a.srcq[q] = src ? static_cast<const char*>(src) + off : nullptr;
    a.dstq[q] = dst ? static_cast<char*>(dst) + off : nullptr;
    a.srci[q] = nullptr;
    a.dsti[q] = nullptr;
    a.lf[q] = a.lb[q] = a.sf[q] = a.sb[q] = 0u;
  }
  return a;
}

// Shifted stream bases of the fast path of periodic pull / AA odd sweeps
// (SweepArgs::srci, dsti); unused by the other kinds.
// Esoteric twist: the read base of direction q is its slot (q even, qbar
// odd) shifted to location x + max(-c_q, 0), the write base its slot (qbar
// even, q odd) shifted to x + max(c_q, 0).
void set_interior(SweepArgs& a, const lbm_ctx* c, int kind) {
  if (kind == K_AA_EVEN) return;
  int32_t cv[27 * 3];
  lbm_stencil_info(c->p.stencil, nullptr, nullptr, cv, nullptr);
  const long long nx = c->p.nx, nxy = (long long)c->p.nx * c->p.ny;
  const long long el = (long long)c->elem;
  auto shift = [](const void* p, long long bytes) {
    return reinterpret_cast<char*>(reinterpret_cast<uintptr_t>(p) + bytes);
  };
  // element offsets of the masked sweeps (SweepArgs::lf, lb, sf, sb)
  const unsigned uN = unsigned(c->N);
  for (int q = 0; q < c->q; ++q) {
    const int cx = cv[3 * q], cy = cv[3 * q + 1], cz = cv[3 * q + 2];
    const int qb = q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1);
    const int lo = q < qb ? q : qb;
    const unsigned e = unsigned(cx + nx * cy + nxy * cz);
    const unsigned w = unsigned(eso_wr(cx) + nx * eso_wr(cy) + nxy * eso_wr(cz));
    auto up = [&](int slot) { return slot != lo ? uN : 0u; };
    if (kind == K_PULL) {
      a.lf[q] = up(q) - e;
      a.lb[q] = up(qb);
    } else if (kind == K_AA_ODD) {
      a.lf[q] = up(qb) - e;
      a.lb[q] = up(q);
      a.sf[q] = up(q) + e;
      a.sb[q] = up(qb);
    } else if (kind == K_ESO_EVEN || kind == K_ESO_ODD) {
      const int sn = kind == K_ESO_EVEN ? qb : q, so = kind == K_ESO_EVEN ? q : qb;
      a.sf[q] = up(sn) + w;
      a.sb[q] = up(so) + w;
    }
  }
  for (int q = 0; q < c->q; ++q) {
    const int cx = cv[3 * q], cy = cv[3 * q + 1], cz = cv[3 * q + 2];
    const long long off = (cx + nx * cy + nxy * cz) * el;
    const int qbar = q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1);
    if (kind == K_ESO_EVEN || kind == K_ESO_ODD) {
      const long long rd = (eso_rd(cx) + nx * eso_rd(cy) + nxy * eso_rd(cz)) * el;
      const long long wr = (eso_wr(cx) + nx * eso_wr(cy) + nxy * eso_wr(cz)) * el;
      a.srci[q] = shift(a.srcq[kind == K_ESO_EVEN ? q : qbar], rd);
      a.dsti[q] = shift(a.dstq[kind == K_ESO_EVEN ? qbar : q], wr);
      continue;
    }
    const int qs = kind == K_AA_ODD ? qbar : q;
    a.srci[q] = shift(a.srcq[qs], -off);
    a.dsti[q] = kind == K_AA_ODD ? shift(a.dstq[q], off) : nullptr;
  }
}

// One time step from state (t, cur) enqueued on stream s.
cudaError_t sweep_once(lbm_ctx* c, cudaStream_t s, int64_t t, int cur) {
  if (c->p.pattern == LBM_PULL) {
    SweepArgs a = make_args(c, c->buf[cur], c->buf[1 - cur]);
    set_interior(a, c, K_PULL);
    if (c->has_mask && c->p.boundary_mode == LBM_BOUNDARY_SEPARATE) {
      const cudaError_t e = c->ops.boundary_pull(a, c->buf[cur], s);
      if (e != cudaSuccess) return e;
    }
    return c->ops.sweep(c->kernel_op, K_PULL, c->has_mask, a, s, c->side_or_null());
  }
  SweepArgs a = make_args(c, c->buf[0], c->buf[0]);
  const bool odd = (t & 1) != 0;
  const int kind = c->p.pattern == LBM_AA ? (odd ? K_AA_ODD : K_AA_EVEN) : (odd ? K_ESO_ODD : K_ESO_EVEN);
  set_interior(a, c, kind);
  return c->ops.sweep(c->kernel_op, kind, c->has_mask, a, s, c->side_or_null());
}

// Records kGraphSteps sweeps starting from pull buffer g (or even parity)
// into c->graph[g].  kGraphSteps is even, so the graph ends in the state
// layout it starts from.
cudaError_t record_graph(lbm_ctx* c, int g) {
  cudaError_t e = cudaSuccess;
  if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  int cur = g;
  for (int i = 0; i < kGraphSteps && le == cudaSuccess; ++i) {
    le = sweep_once(c, c->cap_stream, i, cur);
    cur = 1 - cur;
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[g], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

void drop_graphs(lbm_ctx* c) {
  for (auto& g : c->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

int current_view(const lbm_ctx* c) {
  if (c->p.pattern == LBM_PULL) return V_PULL;
  if (c->p.pattern == LBM_ESOTWIST) return (c->t & 1) ? V_ESO_ODD : V_ESO_EVEN;
  return (c->t & 1) ? V_AA_INVERTED : V_AA_NATURAL;
}

void fill_collide_params(lbm_ctx* c) {
  const lbm_params& p = c->p;
  CollideParams& cp = c->cp;
  std::memset(&cp, 0, sizeof(cp));
  double om[6];
  for (int i = 0; i < 6; ++i) om[i] = p.omega[i];
  if (p.collision == LBM_TRT && p.trt_magic) om[1] = 1.0 / (p.magic / (1.0 / om[0] - 0.5) + 0.5);
  if (p.collision == LBM_MRT && p.stencil != LBM_D3Q27) { om[4] = 1.0; om[5] = 1.0; }
  for (int i = 0; i < 6; ++i) { cp.om_d[i] = om[i]; cp.om[i] = (float)om[i]; }
  if (p.collision == LBM_MRT) {
    if (p.stencil == LBM_D2Q9) mrt_factors<D2Q9>(om, cp);
    else if (p.stencil == LBM_D3Q19) mrt_factors<D3Q19>(om, cp);
    else mrt_factors<D3Q27>(om, cp);
  }
  cp.has_force = (p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0) ? 1 : 0;
  for (int i = 0; i < 3; ++i) { cp.F[i] = p.force[i]; cp.u_wall[i] = p.u_wall[i]; }
  if (c->d == 2) { cp.F[2] = 0.0; cp.u_wall[2] = 0.0; }
  cp.incompressible = p.incompressible ? 1 : 0;
  cp.rho_out = p.rho_outlet;
  cp.smag = p.smagorinsky_cs > 0.0 ? 1 : 0;
  cp.smag_magic = (p.collision == LBM_TRT && p.trt_magic) ? 1 : 0;
  cp.smag_18cs2 = 18.0 * p.smagorinsky_cs * p.smagorinsky_cs;
  cp.smag_tau0 = 1.0 / om[0];
  cp.smag_lambda = p.magic;
  c->kernel_op = p.collision == LBM_KBC ? OP_KBC : p.collision;
  if (cp.smag) c->kernel_op = p.collision == LBM_SRT ? OP_SRT_LES : OP_TRT_LES;
  // MRT whose orders >= 3 share one rate: projector form (collide_mrt3);
  // orders 5 and 6 exist for D3Q27 only
  if (p.collision == LBM_MRT && om[2] == om[3] &&
      (p.stencil != LBM_D3Q27 || (om[4] == om[2] && om[5] == om[2])))
    c->kernel_op = OP_MRT3;
}

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->stencil = LBM_D3Q19;
  p->collision = LBM_TRT;
  p->storage = LBM_F32;
  p->pattern = LBM_PULL;
  p->nx = p->ny = p->nz = 1;
  p->periodic[0] = p->periodic[1] = p->periodic[2] = 1;
  for (int i = 0; i < 6; ++i) p->omega[i] = 1.0;
  p->magic = 3.0 / 16.0;
  p->rho_outlet = 1.0;
}

lbm_status lbm_stencil_info(int32_t stencil, int32_t* q, int32_t* d, int32_t* c, double* w) {
  if (stencil < LBM_D2Q9 || stencil > LBM_D3Q27) return LBM_E_INVAL;
  const int Q = stencil_q(stencil);
  if (q) *q = Q;
  if (d) *d = stencil_d(stencil);
  for (int k = 0; k < Q; ++k) {
    int cx, cy, cz;
    double wk;
    if (stencil == LBM_D2Q9) { cx = D2Q9::cx(k); cy = D2Q9::cy(k); cz = 0; wk = D2Q9::w(k); }
    else if (stencil == LBM_D3Q19) { cx = D3Q19::cx(k); cy = D3Q19::cy(k); cz = D3Q19::cz(k); wk = D3Q19::w(k); }
    else { cx = D3Q27::cx(k); cy = D3Q27::cy(k); cz = D3Q27::cz(k); wk = D3Q27::w(k); }
    if (c) { c[3 * k] = cx; c[3 * k + 1] = cy; c[3 * k + 2] = cz; }
    if (w) w[k] = wk;
  }
  return LBM_OK;
}

lbm_status lbm_query_sizes(const lbm_params* p, size_t* pdf_bytes, size_t* aux_bytes) {
  const char* msg = "";
  const lbm_status s = validate(p, &msg);
  if (s != LBM_OK) return s;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (pdf_bytes) *pdf_bytes = size_t(stencil_q(p->stencil)) * size_t(N) * storage_bytes(p->storage);
  if (aux_bytes) *aux_bytes = layout_for(*p, N).total;
  return LBM_OK;
}

lbm_status lbm_create(lbm_ctx** out, const lbm_params* p, void* pdf, size_t pdf_bytes, void* pdf2,
                      size_t pdf2_bytes, void* aux, size_t aux_bytes, const uint8_t* flags, void* stream) {
  if (!out) return LBM_E_INVAL;
  *out = nullptr;
  const char* msg = "";
  lbm_status s = validate(p, &msg);
  if (s != LBM_OK) return s;
  const long long N = (long long)p->nx * p->ny * p->nz;
  const size_t need = size_t(stencil_q(p->stencil)) * size_t(N) * storage_bytes(p->storage);
  const bool mask = needs_mask(*p, flags != nullptr);
  const Layout lay = layout_for(*p, N);
  if (!pdf || !aux) return LBM_E_INVAL;
  if (p->pattern == LBM_PULL && !pdf2) return LBM_E_INVAL;
  if (pdf_bytes < need || (p->pattern == LBM_PULL && pdf2_bytes < need) || aux_bytes < lay.total)
    return LBM_E_BUFSIZE;
  lbm_ctx* c = injected_alloc_failure() ? nullptr : new (std::nothrow) lbm_ctx;
  if (!c) return LBM_E_NOMEM;
  c->p = *p;
  c->q = stencil_q(p->stencil);
  c->d = stencil_d(p->stencil);
  c->N = N;
  c->elem = storage_bytes(p->storage);
  c->pdf_bytes = need;
  c->aux_bytes = aux_bytes;
  c->buf[0] = pdf;
  c->buf[1] = p->pattern == LBM_PULL ? pdf2 : pdf;
  c->aux = aux;
  c->flags = flags;
  c->has_mask = mask;
  c->mask = mask ? reinterpret_cast<uint32_t*>(static_cast<char*>(aux) + lay.mask_off) : nullptr;
  c->partials = reinterpret_cast<double*>(static_cast<char*>(aux) + lay.part_off);
  c->force_rows = reinterpret_cast<double*>(static_cast<char*>(aux) + lay.adj_off);
  c->result = reinterpret_cast<double*>(static_cast<char*>(aux) + lay.res_off);
  c->stream = static_cast<cudaStream_t>(stream);
  fill_collide_params(c);
  c->ops = get_table(p->stencil, p->storage);
#ifdef LBM_DEBUG_BOUNDS
  if (cudaMemsetAsync(bounds_word(c), 0, sizeof(unsigned), c->stream) != cudaSuccess) {
    delete c;
    return LBM_E_CUDA;
  }
#endif
  if (mask) {
    SweepArgs a = make_args(c, nullptr, nullptr);
    unsigned* types = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(c->result) + 64);
    cudaError_t e = cudaMemsetAsync(types, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = c->ops.link_mask(a, c->mask, types, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&c->link_types, types, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      delete c;
      return LBM_E_CUDA;
    }
    if (p->pattern == LBM_ESOTWIST && (c->link_types & TYPES_FLUID_LAST_LAYER)) {
      delete c;
      return LBM_E_UNSUPPORTED;
    }
    if (p->boundary_mode == LBM_BOUNDARY_SEPARATE &&
        (c->link_types & (TYPES_FLUID_FIRST_LAYER | TYPES_FLUID_LAST_LAYER))) {
      delete c;
      return LBM_E_UNSUPPORTED;
    }
    c->list = reinterpret_cast<uint2*>(static_cast<char*>(aux) + lay.list_off);
    const lbm_status ls = build_list(c, a, lay);
    if (ls != LBM_OK) {
      delete c;
      return ls;
    }
    if (c->n_main > 0 && c->n_wrap > 0) {
      cudaError_t se = cudaStreamCreateWithFlags(&c->side.s, cudaStreamNonBlocking);
      if (se == cudaSuccess) se = cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming);
      if (se == cudaSuccess) se = cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming);
      if (se != cudaSuccess) {
        delete c;
        return LBM_E_CUDA;
      }
    }
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* stream) {
  if (!c) return LBM_E_INVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  return LBM_OK;
}

lbm_status lbm_init_equilibrium(lbm_ctx* c, const double* rho, const double* u) {
  if (!c || !rho || !u) return LBM_E_INVAL;
  c->cur = 0;
  SweepArgs a = make_args(c, nullptr, c->buf[0]);
  cudaError_t e = c->ops.set_state(c->p.pattern, 1, a, nullptr, rho, u, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init_equilibrium");
  c->t = 0;
  return debug_check(c);
}

lbm_status lbm_set_state(lbm_ctx* c, const double* P) {
  if (!c || !P) return LBM_E_INVAL;
  c->cur = 0;
  SweepArgs a = make_args(c, nullptr, c->buf[0]);
  cudaError_t e = c->ops.set_state(c->p.pattern, 0, a, P, nullptr, nullptr, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_state");
  c->t = 0;
  return debug_check(c);
}

lbm_status lbm_step(lbm_ctx* c, int32_t n) {
  if (!c || n < 0) return LBM_E_INVAL;
  const bool graphs = c->N <= kGraphMaxCells;
  while (n > 0) {
    const int g = c->p.pattern == LBM_PULL ? c->cur : 0;
    const bool aligned = c->p.pattern == LBM_PULL || (c->t & 1) == 0;
    if (graphs && aligned && n >= kGraphSteps) {
      cudaError_t e = c->graph[g] ? cudaSuccess : record_graph(c, g);
      if (e == cudaSuccess) e = cudaGraphLaunch(c->graph[g], c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "step graph");
      c->t += kGraphSteps;
      n -= kGraphSteps;
      const lbm_status d = debug_check(c);
      if (d != LBM_OK) return d;
      continue;
    }
    const cudaError_t e = sweep_once(c, c->stream, c->t, c->cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "step");
    if (c->p.pattern == LBM_PULL) c->cur = 1 - c->cur;
    ++c->t;
    --n;
    const lbm_status d = debug_check(c);
    if (d != LBM_OK) return d;
  }
  return LBM_OK;
}

lbm_status lbm_get_time(const lbm_ctx* c, int64_t* t) {
  if (!c || !t) return LBM_E_INVAL;
  *t = c->t;
  return LBM_OK;
}

lbm_status lbm_populations(lbm_ctx* c, double* f) {
  if (!c || !f) return LBM_E_INVAL;
  SweepArgs a = make_args(c, c->buf[c->cur], nullptr);
  cudaError_t e = c->ops.populations(current_view(c), a, f, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "populations");
}

lbm_status lbm_macroscopic(lbm_ctx* c, void* rho, void* u, int32_t out_f64) {
  if (!c || !rho || !u) return LBM_E_INVAL;
  SweepArgs a = make_args(c, c->buf[c->cur], nullptr);
  cudaError_t e = c->ops.macroscopic(current_view(c), a, rho, u, out_f64 != 0, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "macroscopic");
}

lbm_status lbm_reduce(lbm_ctx* c, double out[5]) {
  if (!c || !out) return LBM_E_INVAL;
  SweepArgs a = make_args(c, c->buf[c->cur], nullptr);
  int nb = grid_stride_blocks(c->N, kRedThreads);
  if (nb > kRedMaxBlocks) nb = kRedMaxBlocks;
  cudaError_t e = c->ops.reduce_partial(current_view(c), a, c->partials, nb, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce");
  k_reduce_final<<<1, 32, 0, c->stream>>>(c->partials, nb, c->result);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce");
  e = cudaMemcpyAsync(out, c->result, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce copy");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce sync");
  for (int i = 0; i < 5; ++i)
    if (!std::isfinite(out[i])) {
      set_err(c, "reduction produced a non-finite value");
      return LBM_E_NONFINITE;
    }
  return LBM_OK;
}

lbm_status lbm_get_pdfs(lbm_ctx* c, void* dst) {
  if (!c || !dst) return LBM_E_INVAL;
  cudaError_t e = cudaMemcpyAsync(dst, c->buf[c->cur], c->pdf_bytes, cudaMemcpyDeviceToDevice, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "get_pdfs");
}

lbm_status lbm_set_pdfs(lbm_ctx* c, const void* src, int64_t t) {
  if (!c || !src || t < 0) return LBM_E_INVAL;
  cudaError_t e = cudaMemcpyAsync(c->buf[c->cur], src, c->pdf_bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_pdfs");
  c->t = t;
  return LBM_OK;
}

lbm_status lbm_link_mask(lbm_ctx* c, uint32_t* mask) {
  if (!c || !mask) return LBM_E_INVAL;
  cudaError_t e;
  if (c->has_mask) {
    e = cudaMemcpyAsync(mask, c->mask, size_t(c->N) * 4, cudaMemcpyDeviceToDevice, c->stream);
  } else {
    e = cudaMemsetAsync(mask, 0, size_t(c->N) * 4, c->stream);
  }
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "link_mask");
}

lbm_status lbm_set_force(lbm_ctx* c, const double F[3]) {
  if (!c || !F) return LBM_E_INVAL;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(F[i])) return LBM_E_INVAL;
  if ((c->p.collision == LBM_CUMULANT || c->p.collision == LBM_KBC) && (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0))
    return LBM_E_UNSUPPORTED;
  for (int i = 0; i < 3; ++i) c->p.force[i] = F[i];
  fill_collide_params(c);
  drop_graphs(c);  // recorded sweeps carry the old force
  return LBM_OK;
}

lbm_status lbm_step_pull(lbm_ctx* c, const void* src, void* dst) {
  if (!c || !src || !dst || src == dst) return LBM_E_INVAL;
  if (c->p.pattern != LBM_PULL) return LBM_E_STATE;
  if (c->p.boundary_mode == LBM_BOUNDARY_SEPARATE) return LBM_E_UNSUPPORTED;
  SweepArgs a = make_args(c, src, dst);
  set_interior(a, c, K_PULL);
  cudaError_t e = c->ops.sweep(c->kernel_op, K_PULL, c->has_mask, a, c->stream, c->side_or_null());
  return e == cudaSuccess ? debug_check(c) : cuda_fail(c, e, "step_pull");
}

namespace {
lbm_status adjoint_ok(lbm_ctx* c) {
  if (c->p.pattern != LBM_PULL) {
    set_err(c, "the adjoint works on the two-array pull layout");
    return LBM_E_STATE;
  }
  if (c->p.collision == LBM_CUMULANT || c->p.collision == LBM_KBC) {
    set_err(c, "the cumulant and KBC operators have no adjoint");
    return LBM_E_UNSUPPORTED;
  }
  if (c->link_types & L_OUTLET) {
    set_err(c, "outlet links are not differentiated");
    return LBM_E_UNSUPPORTED;
  }
  if (c->cp.smag) {
    set_err(c, "the Smagorinsky model is not differentiated");
    return LBM_E_UNSUPPORTED;
  }
  if (c->p.boundary_mode == LBM_BOUNDARY_SEPARATE) {
    set_err(c, "the adjoint works with boundary links resolved in the sweep");
    return LBM_E_UNSUPPORTED;
  }
  return LBM_OK;
}
}  // namespace

lbm_status lbm_adjoint_step(lbm_ctx* c, const void* P_prev, const void* lam_in, void* lam_out, double* dLdF) {
  if (!c || !P_prev || !lam_in || !lam_out || lam_in == lam_out) return LBM_E_INVAL;
  lbm_status st = adjoint_ok(c);
  if (st != LBM_OK) return st;
  SweepArgs a = make_args(c, P_prev, nullptr);
  set_interior(a, c, K_PULL);
  // lambda_out bases for the scatter of the periodic fast path: stream q
  // shifted by -c_q (adjoint arrays are FP64 for LBM_F64, FP32 otherwise)
  {
    int32_t cv[27 * 3];
    lbm_stencil_info(c->p.stencil, nullptr, nullptr, cv, nullptr);
    const long long nx = c->p.nx, nxy = (long long)c->p.nx * c->p.ny;
    const long long el = c->p.storage == LBM_F64 ? 8 : 4;
    for (int q = 0; q < c->q; ++q) {
      const long long off = cv[3 * q] + nx * cv[3 * q + 1] + nxy * cv[3 * q + 2];
      a.dsti[q] = reinterpret_cast<char*>(reinterpret_cast<uintptr_t>(lam_out) + (q * c->N - off) * el);
    }
  }
  cudaError_t e = c->ops.adjoint(c->p.collision, c->has_mask, a, lam_in, lam_out, dLdF, c->force_rows, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "adjoint_step");
}

lbm_status lbm_adjoint_segment(lbm_ctx* c, void* const* states, int32_t n, void* lam0, void* lam1, int32_t* cur,
                               double* dLdF) {
  if (!c || !states || n < 1 || !lam0 || !lam1 || lam0 == lam1 || !cur || (*cur != 0 && *cur != 1))
    return LBM_E_INVAL;
  for (int i = 0; i < n; ++i) {
    if (!states[i] || states[i] == lam0 || states[i] == lam1) return LBM_E_INVAL;
    for (int j = 0; j < i; ++j)
      if (states[j] == states[i]) return LBM_E_INVAL;
  }
  lbm_status st = adjoint_ok(c);
  if (st != LBM_OK) return st;
  // recompute P_1 .. P_{n-1} of the segment, then run its adjoint backwards
  for (int i = 1; i < n; ++i) {
    st = lbm_step_pull(c, states[i - 1], states[i]);
    if (st != LBM_OK) return st;
  }
  void* lam[2] = {lam0, lam1};
  int k = *cur;
  for (int t = n; t >= 1; --t) {
    st = lbm_adjoint_step(c, states[t - 1], lam[k], lam[1 - k], dLdF);
    if (st != LBM_OK) return st;
    k = 1 - k;
  }
  *cur = k;
  return LBM_OK;
}

lbm_status lbm_ke_loss_seed(lbm_ctx* c, const void* P, const int32_t box[6], double* L, void* lam_out,
                            double* dLdF) {
  if (!c || !P || !box || !L) return LBM_E_INVAL;
  lbm_status st = adjoint_ok(c);
  if (st != LBM_OK) return st;
  const int32_t n[3] = {c->p.nx, c->p.ny, c->p.nz};
  for (int a = 0; a < 3; ++a)
    if (box[2 * a] < 0 || box[2 * a + 1] > n[a] || box[2 * a] > box[2 * a + 1]) return LBM_E_INVAL;
  SweepArgs a = make_args(c, P, nullptr);
  int b[6];
  for (int i = 0; i < 6; ++i) b[i] = box[i];
  cudaError_t e = c->ops.ke_seed(c->has_mask, a, b, L, lam_out, dLdF, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "ke_loss_seed");
}

lbm_status lbm_eq_vjp(lbm_ctx* c, const double* rho0, const double* u0, const void* lam, double* g_u0) {
  if (!c || !rho0 || !u0 || !lam || !g_u0) return LBM_E_INVAL;
  SweepArgs a = make_args(c, nullptr, nullptr);
  cudaError_t e = c->ops.eq_vjp(a, rho0, u0, lam, g_u0, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "eq_vjp");
}

lbm_status lbm_halo_bytes(const lbm_params* p, size_t* bytes) {
  const char* msg = "";
  const lbm_status s = validate(p, &msg);
  if (s != LBM_OK) return s;
  if (!bytes) return LBM_E_INVAL;
  const int dirs = p->stencil == LBM_D2Q9 ? 3 : (p->stencil == LBM_D3Q19 ? 5 : 9);
  *bytes = size_t(dirs) * size_t(p->ny) * size_t(p->nz) * storage_bytes(p->storage);
  return LBM_OK;
}

namespace {
lbm_status halo(lbm_ctx* c, int32_t face, void* buf, int unpack) {
  if (!c || !buf || (face != LBM_FACE_XLOW && face != LBM_FACE_XHIGH)) return LBM_E_INVAL;
  if (c->p.pattern != LBM_PULL && c->p.pattern != LBM_AA) {
    set_err(c, "block halos are built for the pull and AA patterns");
    return LBM_E_UNSUPPORTED;
  }
  if (c->p.periodic[0] || c->p.nx < 3) {
    set_err(c, "a block needs a non-periodic x axis with ghost layers at x = 0 and nx - 1");
    return LBM_E_INVAL;
  }
  HaloSpec h;
  h.side = face == LBM_FACE_XHIGH ? 1 : 0;
  h.mode = c->p.pattern == LBM_PULL ? 0 : ((c->t & 1) ? 1 : 2);
  h.unpack = unpack;
  SweepArgs a = make_args(c, nullptr, c->buf[c->cur]);
  const cudaError_t e = c->ops.halo(a, h, buf, c->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, unpack ? "halo_unpack" : "halo_pack");
}
}  // namespace

lbm_status lbm_halo_pack(lbm_ctx* c, int32_t face, void* buf) { return halo(c, face, buf, 0); }

lbm_status lbm_halo_unpack(lbm_ctx* c, int32_t face, const void* buf) {
  return halo(c, face, const_cast<void*>(buf), 1);
}

lbm_status lbm_sync(lbm_ctx* c) {
  if (!c) return LBM_E_INVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "sync");
}

const char* lbm_status_str(lbm_status s) {
  if ((int)s < 0 || (int)s > 8) return "LBM_E_UNKNOWN";
  return kStatusNames[(int)s];
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : ""; }

void lbm_debug_fail_host_allocs(int32_t n) { g_fail_allocs.store(n > 0 ? n : 0); }

void lbm_destroy(lbm_ctx* c) { delete c; }

}  // extern "C"
