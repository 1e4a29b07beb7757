// lbm_reduce_noalloc: the FP64 conservation sums of lbm_reduce for callers
// that cannot allocate device memory.
//
// lbm_reduce needs a context, and a context needs a caller-allocated auxiliary
// buffer (link mask and reduction scratch).  Some callers cannot provide one:
// a host application whose device memory belongs to another allocator (a
// framework that reserves the GPU's memory at start-up and forbids further
// cudaMalloc), or a time-step loop that cannot afford cudaMalloc's implicit
// device-wide synchronisation.  This entry point takes the population array
// and flags as they are, derives each cell's boundary links on the fly (with
// the link-mask builder's own per-cell rule, cell_links), and
// keeps its partial sums in a fixed array in the library's own device memory,
// so it allocates nothing.
//
// The scratch is g_partials below: kMaxBlocks rows of 5 doubles (160 KiB).
// The runtime places it on a device when this module is loaded there; with
// lazy module loading (the default of current toolkits) that happens at the
// first call on the device, which can therefore itself take device memory,
// and it stays until the process exits.  Each
// block sums one chunk of kChunk cells, so at most kMaxBlocks * kChunk cells
// (67,108,864) are accepted.  Every call shares the array: a call writes every
// row it later reads, so nothing needs clearing, but two calls that overlap on
// the GPU (for example on two streams) race on it.  The call never
// synchronises, so a non-finite sum is left in out for the caller to test.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

namespace lbm {
namespace noalloc {

constexpr int kThreads = 256;
constexpr long long kChunk = 16384;  // cells per block
constexpr int kMaxBlocks = 4096;
constexpr long long kMaxCells = kChunk * kMaxBlocks;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxBlocks * 5];

// Device address of g_partials per device, looked up once per device with
// that device current.
std::mutex g_lock;
double* g_addr[kMaxDevices] = {};

template <class L, class ST>
__global__ void __launch_bounds__(kThreads) k_partial(const SweepArgs a, int view, double* partials) {
  const long long N = a.g.N;
  const long long begin = blockIdx.x * kChunk;
  const long long end = begin + kChunk < N ? begin + kChunk : N;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long cell = begin + threadIdx.x; cell < end; cell += kThreads) {
    if (a.flags != nullptr && a.flags[cell] != 0) continue;
    int x, y, z;
    cell_coords(a.g, cell, x, y, z);
    unsigned types = 0;
    const uint32_t mask = cell_links<L>(a.g, a.flags, x, y, z, types);
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
  __shared__ double sh[kThreads / 32][5];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < 5; ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) sh[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0;
    for (int w = 0; w < kThreads / 32; ++w) s += sh[w][threadIdx.x];
    partials[blockIdx.x * 5 + threadIdx.x] = s;
  }
}

__global__ void k_final(const double* partials, int nblocks, double* out) {
  if (threadIdx.x < 5) {
    double s = 0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * 5 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

template <class L, class ST>
cudaError_t launch(const SweepArgs& a, int view, double* partials, int nblocks, double* out, cudaStream_t s) {
  k_partial<L, ST><<<nblocks, kThreads, 0, s>>>(a, view, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_final<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

template <class L>
cudaError_t launch_storage(int storage, const SweepArgs& a, int view, double* partials, int nblocks, double* out,
                           cudaStream_t s) {
  switch (storage) {
    case LBM_F64: return launch<L, StF64>(a, view, partials, nblocks, out, s);
    case LBM_F32: return launch<L, StF32>(a, view, partials, nblocks, out, s);
    case LBM_F16S: return launch<L, StF16S>(a, view, partials, nblocks, out, s);
    default: return launch<L, StF32S>(a, view, partials, nblocks, out, s);
  }
}

// Address of g_partials on the current device (set-up on first use).
lbm_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_E_CUDA;
  std::lock_guard<std::mutex> guard(g_lock);
  if (g_addr[dev] == nullptr) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_partials) != cudaSuccess || ptr == nullptr) return LBM_E_CUDA;
    g_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_addr[dev];
  return LBM_OK;
}

}  // namespace noalloc
}  // namespace lbm

extern "C" lbm_status lbm_reduce_noalloc(const lbm_params* p, const void* pdf, const uint8_t* flags, int64_t t,
                                         double* out, void* stream) {
  using namespace lbm;
  if (!p || !pdf || !out || t < 0) return LBM_E_INVAL;
  size_t pdf_bytes = 0;
  lbm_status st = lbm_query_sizes(p, &pdf_bytes, nullptr);
  if (st != LBM_OK) return st;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > noalloc::kMaxCells) return LBM_E_INVAL;  // more cells than the fixed scratch covers
  double* partials = nullptr;
  st = noalloc::scratch_address(&partials);
  if (st != LBM_OK) return st;
  const int q = p->stencil == LBM_D2Q9 ? 9 : (p->stencil == LBM_D3Q19 ? 19 : 27);
  const size_t elem = p->storage == LBM_F64 ? 8 : (p->storage == LBM_F16S ? 2 : 4);
  SweepArgs a{};
  a.src = pdf;
  a.dst = nullptr;
  a.mask = nullptr;
  a.flags = flags;
  a.g.nx = p->nx;
  a.g.ny = p->ny;
  a.g.nz = p->nz;
  for (int i = 0; i < 3; ++i) a.g.per[i] = p->periodic[i] ? 1 : 0;
  if (p->stencil == LBM_D2Q9) a.g.per[2] = 1;
  a.g.N = N;
  for (int k = 0; k < 27; ++k) {
    a.srcq[k] = static_cast<const char*>(pdf) + (k < q ? size_t(k) * size_t(N) * elem : 0);
    a.dstq[k] = nullptr;
  }
  // only the moment parameters matter for the sums
  a.cp.has_force = (p->force[0] != 0.0 || p->force[1] != 0.0 || p->force[2] != 0.0) ? 1 : 0;
  for (int i = 0; i < 3; ++i) {
    a.cp.F[i] = p->force[i];
    a.cp.u_wall[i] = p->u_wall[i];
  }
  if (p->stencil == LBM_D2Q9) { a.cp.F[2] = 0.0; a.cp.u_wall[2] = 0.0; }
  a.cp.incompressible = p->incompressible ? 1 : 0;
  a.cp.rho_out = p->rho_outlet;
  const int view = p->pattern == LBM_PULL       ? V_PULL
                   : p->pattern == LBM_ESOTWIST ? ((t & 1) ? V_ESO_ODD : V_ESO_EVEN)
                                                : ((t & 1) ? V_AA_INVERTED : V_AA_NATURAL);
  const int nblocks = (int)((N + noalloc::kChunk - 1) / noalloc::kChunk);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (p->stencil) {
    case LBM_D2Q9: e = noalloc::launch_storage<D2Q9>(p->storage, a, view, partials, nblocks, out, s); break;
    case LBM_D3Q19: e = noalloc::launch_storage<D3Q19>(p->storage, a, view, partials, nblocks, out, s); break;
    default: e = noalloc::launch_storage<D3Q27>(p->storage, a, view, partials, nblocks, out, s); break;
  }
  return e == cudaSuccess ? LBM_OK : LBM_E_CUDA;
}
