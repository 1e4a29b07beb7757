/*
 * lbm.h -- C ABI of liblbm.so, a GB300 (sm_103a) lattice Boltzmann library.
 *
 * The library implements the fused stream-collide sweep of the lattice
 * Boltzmann method described in Bauer, Koestler & Ruede, "lbmpy: Automatic
 * code generation for efficient parallel lattice Boltzmann methods"
 * (arXiv:2001.11806):
 *   - DdQq stencils D2Q9, D3Q19, D3Q27 (Sec. III-A);
 *   - macroscopic moments rho = sum f, u = sum c f / rho_0 (Eq. density);
 *   - second-order discrete equilibrium (Eq. discrete_eq);
 *   - SRT/BGK (Eq. bgk), TRT (Sec. III-C), MRT with the weighted-orthogonal
 *     moment basis built from the monomial procedure of Sec. III-A (Eq. mrt),
 *     cumulant collision for D3Q27 (Sec. III-B, Eq.
 *     cumulant_generating_function), the Smagorinsky model for SRT/TRT and
 *     the entropic KBC operator (Sec. III-C);
 *   - two-array stream-pull-collide and single-array AA and esoteric-twist
 *     update patterns
 *     (Sec. IV-B "Streaming and Collision");
 *   - per-link boundaries through a flag field (Sec. IV-B "Boundary
 *     Conditions"), compiled into the sweep or, for the two-array pattern,
 *     in a separate boundary kernel: halfway bounce-back, velocity
 *     bounce-back (UBB listing of Sec. III-C) and an equilibrium outlet;
 *   - Guo body forcing (forcing schemes cited in Sec. I);
 *   - a discrete adjoint of the time step (not in the paper).
 * Like the generated kernels of Sec. IV-D, every entry point takes raw
 * pointers, sizes and runtime parameters.
 *
 * Conventions
 *   Cells: x = 0..nx-1 fastest, then y, then z (nz = 1 for D2Q9);
 *     N = nx*ny*nz, cell index n = x + nx*(y + ny*z).
 *   Population arrays: structure of arrays [q][N] in the storage type.
 *   Direction order: 0 is rest; then opposite pairs (2k-1, 2k) as faces
 *     (+x,-x,+y,-y,+z,-z), edges per axis pair xy, xz, yz with signs
 *     (+,+),(-,-),(+,-),(-,+), corners (+++,---), (++-,--+), (+-+,-+-),
 *     (-++,+--).  D2Q9 = rest, 4 faces, 4 xy edges; D3Q19 = rest, faces,
 *     edges; D3Q27 = D3Q19 + corners.  lbm_stencil_info returns the table.
 *   State: the library's canonical state P is the post-collision populations
 *     of the last completed step (two-array pull convention).  A step is
 *     f_q(x) = P_q(x - c_q) if x - c_q is fluid, else B_q(P(x)) (boundary
 *     link), then P'(x) = collide(f(x)) on fluid cells.  Initialisation sets
 *     P = f^eq(rho_0, u_0).  "Populations" are the streamed f of the current
 *     time; macroscopic output and reductions are moments of them.
 *   Shifted storage (LBM_F32S, LBM_F16S) stores h_q = f_q - w_q.
 *
 * Ownership: the caller allocates and owns every device buffer (for example
 *   with torch); the library borrows pointers and never frees them.  A
 *   context owns host metadata only.  Buffers must stay valid until
 *   lbm_destroy.
 * Asynchrony: calls enqueue work on the context's CUDA stream and return;
 *   lbm_reduce and lbm_sync synchronise the stream.
 * Errors: every call returns lbm_status; none throws, exits or traps.
 *   Invalid arguments are rejected before any launch.  A CUDA error after a
 *   launch returns LBM_E_CUDA; lbm_last_error gives the message.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lbm_status {
  LBM_OK = 0,
  LBM_E_INVAL = 1,       /* bad argument or parameter value */
  LBM_E_UNSUPPORTED = 2, /* valid but not built (e.g. cumulant on D2Q9) */
  LBM_E_CUDA = 3,        /* a CUDA runtime call or launch failed */
  LBM_E_NOMEM = 4,       /* host allocation failed */
  LBM_E_BUFSIZE = 5,     /* a caller buffer is smaller than required */
  LBM_E_NONFINITE = 6,   /* a reduction found NaN or Inf */
  LBM_E_BOUNDS = 7,      /* a kernel addressed memory outside the population arrays;
                          * only a library built with LBM_DEBUG_BOUNDS checks this
                          * (lbm_init_equilibrium, lbm_set_state, lbm_step and
                          * lbm_step_pull then synchronise and report it) */
  LBM_E_STATE = 8        /* call not valid in the current state */
} lbm_status;

enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 };
/* LBM_KBC: entropic KBC (Sec. III-C, Eq. entropic_linear_update and
 * Eq. entropic_direct_omega_eq), the rate of the moments of order >= 3 chosen
 * per cell and step from the linearised entropy condition */
enum { LBM_SRT = 0, LBM_TRT = 1, LBM_MRT = 2, LBM_CUMULANT = 3, LBM_KBC = 4 };
/* storage type of the population arrays; the collision computes in FP64 for
 * LBM_F64 and in FP32 for the others */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_F32S = 3 };
/* update pattern (Sec. IV-B "Streaming and Collision"):
 *   LBM_PULL: two arrays, stream-pull-collide, swapped every step;
 *   LBM_AA: one array; even steps read and write a cell's own slots, odd
 *     steps read and write its neighbours';
 *   LBM_ESOTWIST: one array; every step reads and writes the slots at the
 *     cell and at its positive neighbours x + max(c_q, 0): f_q(x) is read from
 *     location x + max(-c_q, 0) (slot q after an even number of steps, slot
 *     qbar after an odd number) and P_q(x) written to x + max(c_q, 0) (slot
 *     qbar in even steps, q in odd steps; a boundary link (x, qbar) takes the
 *     other slot).  Locations wrap on every axis, so along a non-periodic
 *     axis the last layer (index n - 1) must be non-fluid (a wall, inlet or
 *     outlet layer); lbm_create returns LBM_E_UNSUPPORTED otherwise. */
enum { LBM_PULL = 0, LBM_AA = 1, LBM_ESOTWIST = 2 };
enum { LBM_BOUNDARY_IN_SWEEP = 0, LBM_BOUNDARY_SEPARATE = 1 };
/* uint8 flag per cell; 0 = fluid.  A boundary link (x, q) takes its type from
 * the flag of its source cell x - c_q with precedence NOSLIP > INLET > OUTLET
 * (a non-zero flag with none of these bits and without the GHOST bit counts as
 * NOSLIP).  Sources outside a non-periodic axis count as NOSLIP.
 * GHOST (without NOSLIP, INLET or OUTLET; other bits ignored): a ghost cell of
 * a block partition (Sec. IV-D "Framework Integration"): it is not swept and
 * its populations come from the neighbouring block (lbm_halo_unpack), and
 * links from it stream like fluid links. */
enum { LBM_FLUID = 0, LBM_NOSLIP = 1, LBM_INLET = 2, LBM_OUTLET = 4, LBM_GHOST = 8 };
/* bit 31 of a link-mask word marks a non-fluid cell; bit 30 marks a fluid
 * cell that has at least one INLET or OUTLET link; bit 29 (with bit 31) marks
 * a ghost cell */
#define LBM_MASK_SOLID 0x80000000u
#define LBM_MASK_SPECIAL 0x40000000u
#define LBM_MASK_GHOST 0x20000000u

typedef struct lbm_params {
  int32_t stencil;      /* LBM_D2Q9 | LBM_D3Q19 | LBM_D3Q27 */
  int32_t collision;    /* LBM_SRT | LBM_TRT | LBM_MRT | LBM_CUMULANT | LBM_KBC */
  int32_t storage;      /* LBM_F64 | LBM_F32 | LBM_F16S | LBM_F32S */
  int32_t pattern;      /* LBM_PULL | LBM_AA | LBM_ESOTWIST */
  int32_t nx, ny, nz;   /* nz must be 1 for D2Q9; each >= 1 */
  int32_t periodic[3];  /* non-zero = periodic along x, y, z */
  /* relaxation rates, each in (0, 2):
   *   SRT: omega[0] = omega.
   *   TRT: omega[0] = omega_e (even moments), omega[1] = omega_o (odd).
   *   MRT: shear, bulk, 3rd-order, 4th-order, 5th-order, 6th-order rates
   *        (orders 5 and 6 exist for D3Q27 only); conserved moments use 0.
   *        When all orders >= 3 share one rate the sweep uses an equivalent
   *        projector form of the operator (same result up to rounding).
   *   CUMULANT: shear, bulk, higher-order (orders >= 3).
   *   KBC: omega[0] = shear rate omega_s, omega[1] = bulk rate (equal to
   *        omega[0] gives the paper's two-rate form); the rate of orders >= 3
   *        is not a parameter.  No body force, no Smagorinsky model. */
  double omega[6];
  int32_t trt_magic;    /* TRT: non-zero derives omega_o from omega_e and Lambda = magic */
  int32_t incompressible; /* non-zero: rho_0 = 1 in velocity terms (Sec. III-A) */
  double magic;         /* Lambda = (1/omega_e - 1/2)(1/omega_o - 1/2), e.g. 3/16 */
  double u_wall[3];     /* velocity of INLET (UBB) links, rho_0 = 1 */
  double rho_outlet;    /* density of OUTLET links: B_q = f^eq_q(rho_outlet, u_P(x)) */
  double force[3];      /* uniform body force, Guo scheme; zero = no force */
  /* Smagorinsky constant C_S (filter width 1) for SRT/TRT; 0 = off.  The even
   * rate becomes a per-cell omega from the non-equilibrium stress (Sec. III-C,
   * turbulence models); with trt_magic the odd rate follows through Lambda. */
  double smagorinsky_cs;
  /* LBM_BOUNDARY_IN_SWEEP (default): boundary links are resolved inside the
   * sweep through the link mask.  LBM_BOUNDARY_SEPARATE (two-grid pull
   * only): before every sweep a boundary kernel writes B_q(P(x)) into the
   * slot of the link's non-fluid source cell, and the sweep streams every
   * link as if it were fluid (Sec. IV-B "Boundary Conditions", the variant
   * with separate boundary kernels).  Every boundary-link source must then
   * lie inside the box: along a non-periodic axis the first and the last
   * layer must be non-fluid (LBM_E_UNSUPPORTED otherwise, or for AA and the
   * esoteric twist). */
  int32_t boundary_mode;
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Fill *p with defaults: D3Q19 TRT FP32 pull, 1^3 periodic cells, omega 1.0,
 * rho_outlet 1, no force.  Interface plumbing (the runtime parameters of
 * Sec. IV-D), no method step of its own. */
void lbm_default_params(lbm_params* p);

/* Stencil table of the DdQq velocity sets and weights (Sec. III-A, c_s^2 =
 * 1/3): *q, *d, and if non-NULL c[q*3] (integer velocities, unused
 * components zero) and w[q] (weights).  Returns LBM_E_INVAL for an unknown
 * stencil. */
lbm_status lbm_stencil_info(int32_t stencil, int32_t* q, int32_t* d, int32_t* c, double* w);

/* Bytes the caller must allocate (the array layout that Sec. IV-D passes as
 * shape and stride, q values per cell as counted in Sec. V): pdf_bytes for
 * each population array (q * N * sizeof(storage)); aux_bytes for the auxiliary device buffer
 * (link mask of 4*N bytes and fluid-cell list of 8*N bytes, used when flags
 * or non-periodic axes are present but reserved in every case, the list
 * builder's counts and the reduction scratch).  Validates p. */
lbm_status lbm_query_sizes(const lbm_params* p, size_t* pdf_bytes, size_t* aux_bytes);

/* Create a context over caller-owned device buffers (Sec. IV-D "Framework
 * Integration": each generated kernel takes raw array pointers, the shape
 * that fixes their layout, and the method's free symbols, relaxation rates
 * and forces, as runtime parameters; here they are gathered once in p).
 *   pdf, pdf2: population arrays of pdf_bytes each; pdf2 must be non-NULL for
 *     LBM_PULL and is ignored (may be NULL) for LBM_AA and LBM_ESOTWIST.
 *   aux: auxiliary device buffer of aux_bytes.
 *   flags: device uint8[N] flag field or NULL (all fluid).  It is read at
 *     creation (to build the link mask) and on boundary links during steps.
 *   stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 * Byte sizes are checked against lbm_query_sizes (LBM_E_BUFSIZE).  The
 * populations are undefined until lbm_init_equilibrium or lbm_set_state. */
lbm_status lbm_create(lbm_ctx** out, const lbm_params* p, void* pdf, size_t pdf_bytes,
                      void* pdf2, size_t pdf2_bytes, void* aux, size_t aux_bytes,
                      const uint8_t* flags, void* stream);

/* Change the stream later calls enqueue on (interface plumbing, no method
 * step; the paper's GPU kernels run on pycuda streams, Sec. IV-D). */
lbm_status lbm_set_stream(lbm_ctx* ctx, void* stream);

/* Set P = f^eq(rho_0, u_0) (Eq. discrete_eq, second order) from device FP64 arrays
 * rho[N] and u[d][N]; resets the step counter to 0. */
lbm_status lbm_init_equilibrium(lbm_ctx* ctx, const double* rho, const double* u);

/* Set P from a device FP64 array P[q][N] (unshifted populations), written
 * in the pattern's layout (Sec. IV-B "Streaming and Collision"); resets the
 * step counter to 0. */
lbm_status lbm_set_state(lbm_ctx* ctx, const double* P);

/* Advance n >= 0 time steps (asynchronous).  One step is the fused
 * stream-collide sweep of Sec. IV-B "Streaming and Collision" in the
 * configured pattern (two-array pull, AA or esoteric twist), with the
 * boundary links of Sec. IV-B "Boundary Conditions" resolved in the sweep
 * or, for LBM_BOUNDARY_SEPARATE, by a boundary kernel run before it. */
lbm_status lbm_step(lbm_ctx* ctx, int32_t n);

/* Number of steps since the last initialisation (AA and esoteric-twist parity
 * = t mod 2, Sec. IV-B "Streaming and Collision": the single-array patterns
 * alternate between an even and an odd kernel). */
lbm_status lbm_get_time(const lbm_ctx* ctx, int64_t* t);

/* Populations f of the current time (streamed, pre-collision, unshifted) as
 * device FP64 f[q][N], read through the pattern's current parity (Sec. IV-B
 * "Streaming and Collision"); non-fluid cells are written as NaN. */
lbm_status lbm_populations(lbm_ctx* ctx, double* f);

/* rho[N] and u[d][N] (device, FP64 if out_f64 else FP32) from the current
 * populations: rho = sum f, u = (sum c f + F/2) / rho_0 (Eq. density with the
 * Guo half force).  Non-fluid cells are written as NaN. */
lbm_status lbm_macroscopic(lbm_ctx* ctx, void* rho, void* u, int32_t out_f64);

/* FP64 sums over fluid cells: out[0] = sum rho, out[1..3] = sum rho_0 u,
 * out[4] = (1/2) sum rho |u|^2.  Host array out[5].  Synchronises the
 * stream.  Returns LBM_E_NONFINITE if any sum is NaN or Inf.  Not in the
 * paper: a conservation check built on its statement that collisions
 * conserve mass and momentum (Sec. III-A, the conserved moments of rate 0),
 * with moments as in Eq. density. */
lbm_status lbm_reduce(lbm_ctx* ctx, double out[5]);

/* Raw copy of the native population storage (pdf_bytes, device to device),
 * for checkpoint/restore.  lbm_set_pdfs also sets the step counter to t so
 * that the AA or esoteric-twist parity matches the saved data.  Not in the
 * paper: the saved layout is the pattern's own (Sec. IV-B "Streaming and
 * Collision"), so a restore needs the step parity with it. */
lbm_status lbm_get_pdfs(lbm_ctx* ctx, void* dst);
lbm_status lbm_set_pdfs(lbm_ctx* ctx, const void* src, int64_t t);

/* Device uint32[N] link mask: bit q set when the source x - c_q of a fluid
 * cell x is not fluid (a boundary link); LBM_MASK_SPECIAL when one of those
 * links is an INLET or OUTLET link; LBM_MASK_SOLID for non-fluid cells.
 * Computed on the device from the flags.  This is the per-cell form of the
 * paper's per-link boundary information (Sec. IV-B "Boundary Conditions":
 * a flag field sets up the boundaries, from which one entry per boundary
 * link is extracted); exported for bit-exact checks of that extraction. */
lbm_status lbm_link_mask(lbm_ctx* ctx, uint32_t* mask);

/* Replace the uniform body force (Guo scheme, Sec. I; like the paper's
 * constant external forces it is a runtime parameter of the kernels, Sec.
 * IV-D); takes effect for later launches.  LBM_E_UNSUPPORTED for a non-zero force with cumulant or KBC
 * collision. */
lbm_status lbm_set_force(lbm_ctx* ctx, const double F[3]);

/* One time step of the pull pattern from the population array src into dst
 * (both pdf_bytes, distinct; the context's own arrays are not touched): the
 * two-array stream-pull-collide sweep of Sec. IV-B "Streaming and Collision"
 * on explicit arrays.  LBM_E_STATE for an AA context, LBM_E_UNSUPPORTED with
 * separate boundary kernels.  Not a separate step of the paper: it exists to
 * recompute checkpoint segments for the adjoint. */
lbm_status lbm_step_pull(lbm_ctx* ctx, const void* src, void* dst);

/* Discrete adjoint of one pull time step (the paper has no adjoint; this is
 * the reverse-mode derivative of the sweep): lam_out = S^T C'(f)^T lam_in,
 * with f = S(P_prev) the populations the forward step collided (S = pull
 * streaming with boundary links, C = collision).  If dLdF is non-NULL, the
 * body-force gradient of the step, sum_x (dC/dF)^T lam_in, is added to the
 * device double[3] it points to.  lam_in, lam_out: device [q][N] arrays of FP64
 * when storage is LBM_F64, else FP32 (distinct).  P_prev: device population
 * array in the storage type.  Requires the pull pattern (LBM_E_STATE), SRT,
 * TRT or MRT without the Smagorinsky model (LBM_E_UNSUPPORTED for cumulant,
 * KBC and Smagorinsky), boundary links resolved in the sweep and no OUTLET
 * links (LBM_E_UNSUPPORTED).  Non-fluid cells receive zero. */
lbm_status lbm_adjoint_step(lbm_ctx* ctx, const void* P_prev, const void* lam_in, void* lam_out,
                            double* dLdF);

/* Reverse sweep of one checkpoint segment of n >= 1 steps, enqueued from the
 * library so that no per-step host round trip is needed (not in the paper:
 * the schedule of the sqrt(T) checkpointing the adjoint uses).
 *   states: host array of n distinct device population arrays (pdf_bytes
 *     each, storage type); states[0] holds the checkpoint P_s, states[1 ..
 *     n-1] receive the recomputed P_{s+1} .. P_{s+n-1} (one lbm_step_pull
 *     each);
 *   lam0, lam1: the two adjoint arrays of lbm_adjoint_step (distinct, and
 *     distinct from every state); *cur (0 or 1) names the one holding
 *     lambda_{s+n} on entry and, on return, the one holding lambda_s;
 *   dLdF: as in lbm_adjoint_step (accumulated over the n steps) or NULL.
 * Then for t = s + n down to s + 1: lambda_{t-1} = adjoint_step(P_{t-1},
 * lambda_t).  Same requirements and errors as lbm_step_pull and
 * lbm_adjoint_step; LBM_E_INVAL for aliased buffers. */
lbm_status lbm_adjoint_segment(lbm_ctx* ctx, void* const* states, int32_t n, void* lam0, void* lam1, int32_t* cur,
                               double* dLdF);

/* Not in the paper (the objective of the adjoint): kinetic energy in a box,
 * L = (1/2) sum rho |u|^2 over the fluid cells with
 * box[0] <= x < box[1], box[2] <= y < box[3], box[4] <= z < box[5], of the
 * populations f = S(P) (u with the Guo half force), ADDED to the device
 * double *L.  If lam_out is non-NULL it receives the adjoint seed
 * S^T dL/df (layout and type as in lbm_adjoint_step); if dLdF is non-NULL the
 * explicit body-force derivative of L is added to it.  Same requirements as
 * lbm_adjoint_step. */
lbm_status lbm_ke_loss_seed(lbm_ctx* ctx, const void* P, const int32_t box[6], double* L, void* lam_out,
                            double* dLdF);

/* g_u0 = (d f^eq(rho_0, u_0) / d u_0)^T lam for the initial state written by
 * lbm_init_equilibrium: rho0[N], u0[d][N] and g_u0[d][N] are device FP64, lam
 * as in lbm_adjoint_step.  Non-fluid cells receive zero.  Not in the paper:
 * the transpose of the derivative of Eq. discrete_eq with respect to u,
 * which closes the adjoint sweep at t = 0. */
lbm_status lbm_eq_vjp(lbm_ctx* ctx, const double* rho0, const double* u0, const void* lam, double* g_u0);

/* The sums of lbm_reduce without a context and without any allocation, for
 * callers that cannot allocate device memory: for example a host application
 * whose GPU memory belongs to another allocator that reserves it at start-up,
 * or a time-step loop that cannot afford cudaMalloc's implicit device-wide
 * synchronisation.  The paper has no counterpart; it exists for such callers.
 *   p:      the parameters the populations were produced with (validated as in
 *           lbm_query_sizes);
 *   pdf:    device population array in the native layout, as lbm_get_pdfs
 *           returns it (for LBM_PULL the array holding the current state);
 *   flags:  device uint8[N] flag field or NULL (all fluid);
 *   t:      the step count of that state (selects the AA / esoteric-twist parity);
 *   out:    device double[5]; receives the same five sums as lbm_reduce;
 *   stream: cudaStream_t (NULL = legacy default stream); the call enqueues work
 *           and returns without synchronising.
 * Scratch lives in a fixed 160 KiB array in the library's device memory.  The
 * CUDA runtime places it on a device when the library's module is loaded
 * there, which with lazy module loading (the default of current toolkits) is
 * the first call on that device, not the loading of the library: that first
 * call (with the device current) loads the module, places the array and looks
 * up its device address, so it can itself take 160 KiB of device memory and
 * fail with LBM_E_CUDA if none is left.  Callers whose allocator reserves the
 * GPU should therefore make one call at start-up, before the allocator takes
 * the memory, and before any stream capture.  The array then stays until the
 * process exits.  Every call shares it: calls that overlap on the GPU race.
 * The call does not synchronise, so it cannot report a non-finite sum
 * (lbm_reduce's LBM_E_NONFINITE): a NaN or Inf is left in out, and a caller
 * using the sums as a conservation check must test out[] after synchronising.
 * Returns LBM_E_INVAL for more than 67,108,864 cells (the cells the fixed
 * scratch covers), and never calls cudaMalloc or cudaFree. */
lbm_status lbm_reduce_noalloc(const lbm_params* p, const void* pdf, const uint8_t* flags, int64_t t,
                              double* out, void* stream);

/* Halo exchange of x-slab blocks (Sec. IV-D "Framework Integration": a
 * block-structured domain partition, with pack and unpack kernels for the
 * communication between blocks, generated there because for the single-array
 * patterns which values cross a face depends on the step parity).
 * A block is a context whose x axis is not periodic, with one ghost layer at
 * x = 0 and x = nx - 1: flag LBM_GHOST where the neighbouring block's cell is
 * fluid, its own flag otherwise (NOSLIP outside a non-periodic global
 * domain); y and z are the global domain's.  After lbm_init_equilibrium /
 * lbm_set_state and after every step, each block packs what crosses each of
 * its faces (lbm_halo_pack) and its neighbour across that face unpacks it
 * (lbm_halo_unpack of the opposite face) before the next step; the blocks
 * then step like one domain, bit for bit.  Pull and AA patterns only
 * (LBM_E_UNSUPPORTED otherwise); LBM_E_INVAL for a periodic x axis or
 * nx < 3.
 *   face: LBM_FACE_XLOW (x = 0) or LBM_FACE_XHIGH (x = nx - 1);
 *   buf:  device buffer of lbm_halo_bytes: the crossing directions' values
 *         ([k][z][y] in the storage type, k over the directions with
 *         c_x = +1 for XHIGH packs and XLOW unpacks, c_x = -1 otherwise).
 *         An unpack leaves the receiver's own boundary values in place (links
 *         whose source across the face is not fluid).
 * Asynchronous on the context's stream. */
enum { LBM_FACE_XLOW = 0, LBM_FACE_XHIGH = 1 };
lbm_status lbm_halo_bytes(const lbm_params* p, size_t* bytes);
lbm_status lbm_halo_pack(lbm_ctx* ctx, int32_t face, void* buf);
lbm_status lbm_halo_unpack(lbm_ctx* ctx, int32_t face, const void* buf);

/* Block until the context's stream is idle; maps pending CUDA errors
 * (interface plumbing, no method step). */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Name of a status code; lbm_last_error: last error message of this context
 * ("" if none), never NULL.  Error reporting of the interface, no method
 * step. */
const char* lbm_status_str(lbm_status s);
const char* lbm_last_error(const lbm_ctx* ctx);

/* Test hook for the failure paths (the paper has no counterpart): the next n
 * host allocations made by the library fail, so that the calls making them
 * return LBM_E_NOMEM (lbm_create allocates its context; a context with a
 * flag field also allocates the offsets of its fluid-cell list).  n <= 0
 * clears the request.  Process-wide, not thread-specific. */
void lbm_debug_fail_host_allocs(int32_t n);

/* Free the context's host metadata; device buffers stay the caller's.
 * Interface plumbing, no method step. */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
