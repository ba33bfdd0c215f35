/*
 * lbm.h -- C ABI of the GB300 two-component lattice Boltzmann library (liblbm.so).
 *
 * The library advances one lattice of either model compared in arXiv 2110.05197
 * (Datadien, Di Staso, Wijshoff & Toschi):
 *   - the colour-gradient (CG) model of Sec. 2.2: two population sets (red, blue), BGK
 *     towards the enhanced equilibrium (Eq. equiliCG), the surface-tension perturbation
 *     (Eq. perturbationOp), recolouring (Eqs. recoloringOpR/B), optionally the
 *     inter-interface repulsion force of Sec. 2.3 (Eq. repForce), then streaming
 *     (Eq. streaming);
 *   - the Shan-Chen (SC) model of Sec. 2.1: the multiphase pseudopotential force
 *     (Eqs. interactionforceMP, pseudopotential) or the two-component cross force
 *     (Eq. doublebeltrepulsionforce2), Guo forcing (Eqs. guoforce, source, guoforce2),
 *     BGK (Eqs. collisSC, equiliSC), streaming (Eq. streamingSC).
 * The problem statement the calls follow is the paper's: initialise the component
 * densities (and velocity) on a periodic box (Sec. 3), evolve a number of steps, measure
 * moments (Sec. 3.1, Eqs. YoungLaplace..rhoout; Sec. 3.2).
 *
 * Conventions
 *   - Every call returns an lbm_status; nothing is thrown across the ABI.  After a CUDA
 *     error the context keeps the first error (sticky) and every later call returns it.
 *   - The caller owns all device memory and the stream.  lbm_create only reports the
 *     workspace size it needs (ws == NULL) or binds the caller's workspace; the library
 *     never allocates device memory.  The context object itself is a small host struct.
 *   - All device work is enqueued on the stream given to lbm_create.  Calls return without
 *     synchronising, except where a host pointer is read or written (see below).
 *   - Lattice layout: node = x + nx*(y + ny*z), x fastest.  Populations are
 *     structure-of-arrays [component][direction][node].  Direction order (the paper lists
 *     only the groups, Eq. speeds):
 *       D3Q19: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),(-1,-1,0),(1,-1,0),
 *              (-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),
 *              (0,-1,1);
 *       D2Q9:  0 rest; 1..4 = +x,-x,+y,-y; 5..8 = (1,1),(-1,-1),(1,-1),(-1,1).
 *     The opposite of odd direction i >= 1 is i+1.
 *   - Pointer arguments of lbm_init_fields and lbm_moments may be device pointers or host
 *     pointers (pinned or pageable); the library inspects each one.  Host data is staged
 *     through the workspace with cudaMemcpyAsync on the context's stream; a call that reads
 *     or writes a host pointer synchronises that stream before returning.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,     /* bad argument: NULL where required, size or parameter out of range */
  LBM_ENOMEM = 2,     /* workspace smaller than lbm_create reported */
  LBM_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed (sticky) */
  LBM_EUNSTABLE = 4,  /* the blow-up check tripped: non-finite, negative density or |u| too large */
  LBM_ESTATE = 5,     /* call does not fit the context: wrong model for this step call, or
                         stepping before lbm_init_fields */
  LBM_ETIMEOUT = 6    /* a step kernel's bounded device wait gave up (2 s of GPU time on one
                         wait) or its shared-memory layout check failed; the state stops
                         advancing and lbm_moments(totals) reports this status */
} lbm_status;

enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };
enum { LBM_MODEL_CG = 0, LBM_MODEL_SC_MP = 1, LBM_MODEL_SC_2C = 2, LBM_MODEL_SC_MR = 3 };
/* Storage precision of the populations.  FP64 computes in FP64; the others compute in FP32.
 * Populations are stored as deviations from the rest-state equilibrium of each node's
 * density one step earlier (kept in a reference field, FP64 for LBM_FP64, FP32 otherwise),
 * so 16-bit storage holds only the small non-equilibrium and velocity parts. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16 = 2, LBM_BF16 = 3 };
/* Streaming storage (Eq. streaming).  LBM_STREAM_AB: two population buffers, the step reads
 * one and pushes into the other.  LBM_STREAM_AA: one buffer updated in place (AA pattern:
 * even steps write each node's post-collision populations back into its own slots, reversed;
 * odd steps read from and write to the neighbours' slots), which halves the population
 * memory; each step then also runs a field pass over the populations (densities and
 * stencil fields of time t, which the in-place update would otherwise overwrite), so it
 * moves about 1.5x the bytes.  Results agree with LBM_STREAM_AB to rounding. */
enum { LBM_STREAM_AB = 0, LBM_STREAM_AA = 1 };
enum { LBM_NTOTALS = 10 };

/* Parameters of one lattice.  Field meanings follow the paper's notation. */
typedef struct {
  int32_t lattice;        /* LBM_D2Q9 (nz must be 1) or LBM_D3Q19 */
  int32_t model;          /* LBM_MODEL_CG, LBM_MODEL_SC_MP (one set), LBM_MODEL_SC_2C (two sets),
                             LBM_MODEL_SC_MR (two sets, multirange potentials; D3Q19 only) */
  int32_t precision;      /* LBM_FP64, LBM_FP32, LBM_FP16 or LBM_BF16 (see above) */
  int32_t nx, ny, nz;     /* lattice size, each >= 1; periodic in every direction */
  double rho_r0, rho_b0;  /* CG bulk densities; density ratio gamma = rho_r0/rho_b0 (Eq. gamma) */
  double alpha_b;         /* CG rest parameter of the blue fluid (0.2 in the paper); alpha_R from
                             Eq. gamma */
  double tau_r, tau_b;    /* relaxation times (> 1/2); nu_k = (tau_k - 1/2)/3; SC multiphase
                             uses tau_r */
  double A, beta;         /* CG perturbation amplitude (sigma = 4/9 A/omega_eff, Eq. sigmaA) and
                             recolouring parameter (0.7 in the paper) */
  int32_t enhanced_eq;    /* 1: enhanced equilibrium of Eq. equiliCG; 0: its plain second-order
                             part (the "standard" CG of Sec. 3.3) */
  int32_t color_norm;     /* 0: rho^N = (rho_R - rho_B)/(rho_R + rho_B) as printed; 1: each
                             density divided by its bulk value rho_k0 first */
  double rep_pi, rep_chi; /* CG repulsion: Pi (0 disables the force) and chi (Eq. potential) */
  int32_t rep_psi_kind;   /* 0: psi_rep = (1 - |rho^N|)^chi; 1: (1 + |rho^N|)^chi as printed */
  double grad_eps;        /* |grad rho^N| <= grad_eps: no perturbation, cos(phi_i) = 0, no normal */
  double G, rho0_psi;     /* SC coupling G and reference density rho_0 (multiphase psi) or
                             rho_0^(s) (two-component cross force) */
  double body_force[3];   /* constant body-force density (Guo forcing); 0 for none */
  int32_t diag_every;     /* run the blow-up check every n steps inside lbm_step_*; 0 = never */
  double umax_unstable;   /* blow-up threshold on |u| (default used when <= 0: 0.5) */
  int32_t streaming;      /* LBM_STREAM_AB (0, default) or LBM_STREAM_AA (see above) */
  double Ga[2], Gr[2];    /* LBM_MODEL_SC_MR (Sec. 2.1, Eq. benziforces): per species the
                             attractive belt-1 coupling G^a (lattice weights w, Eq.
                             doublebeltattractiveforce) and the repulsive belts-1+2 coupling
                             G^r (weights p of Eq. pweights over the 92 vectors with
                             |c|^2 <= 8, Eq. doublebeltrepulsionforce), acting on
                             Psi_s = rho0_psi (1 - exp(-rho_s / rho0_psi)); G is the cross
                             coupling G_AB of Eq. doublebeltrepulsionforce2.  The model steps
                             with lbm_step_sc on the field-pass kernels (its force reaches
                             distance 2), in either streaming mode; the batched launch and
                             lbm_totals_noalloc do not take it. */
} lbm_params;

/* Validate p and size the workspace.
 *   ws == NULL: write the required workspace size (bytes) to *ws_bytes and return LBM_OK;
 *               *out is left untouched.
 *   ws != NULL: ws must be a device buffer of at least the required size, 256-byte aligned,
 *               owned by the caller and kept alive until lbm_destroy; *ws_bytes gives its
 *               size (LBM_ENOMEM if too small).  Creates the context in *out.
 * stream is a cudaStream_t (NULL = legacy default stream) on which all work is enqueued.
 * Errors: LBM_EINVAL for NULL p/ws_bytes/out or parameters out of range. */
lbm_status lbm_create(const lbm_params* p, void* ws, size_t* ws_bytes, void* stream, lbm_ctx** out);

/* Set the initial state (Sec. 3: sharp-interface component densities, optional velocity).
 *   rho_r [N]: density of component R (CG red / SC multiphase rho / SC species 1); required.
 *   rho_b [N]: density of component B (CG blue / SC species 2); ignored for SC multiphase.
 *   u [3][N] (component-major), solid [N] (uint8, 1 = wall node), pops [K][Q][N]: optional.
 * All floating-point inputs are FP64.  With pops != NULL the populations are taken from it
 * (checkpoint restore, canonical order, rho_r/rho_b/u unused but rho_r must be non-NULL);
 * otherwise f^k = f^{k,eq}(rho_k, u, grad rho_k) (CG, Eq. equiliCG) or f^eq(rho_s, u)
 * (SC, Eq. equiliSC).  Wall nodes hold no populations.  Resets the step counter and the
 * blow-up status.  Reads host pointers synchronously. */
lbm_status lbm_init_fields(lbm_ctx* ctx, const double* rho_r, const double* rho_b, const double* u,
                           const uint8_t* solid, const double* pops);

/* Advance nsteps (>= 0) colour-gradient steps.  LBM_ESTATE if the model is not CG or the
 * fields were never initialised.  Asynchronous. */
lbm_status lbm_step_cg(lbm_ctx* ctx, int32_t nsteps);

/* Advance nsteps (>= 0) Shan-Chen steps (multiphase or two-component, by model).
 * LBM_ESTATE if the model is CG or the fields were never initialised.  Asynchronous. */
lbm_status lbm_step_sc(lbm_ctx* ctx, int32_t nsteps);

/* Moments of the current state.  Every output may be NULL.  Outputs are FP64:
 *   rho_r, rho_b [N]; u [3][N] = (sum_k sum_i f c_i + F/2)/rho, the force-shifted velocity of
 *   Eq. guoforce (0 on wall nodes); pops [K][Q][N] canonical post-streaming populations;
 *   totals (HOST, LBM_NTOTALS doubles): mass_r, mass_b, momentum x/y/z (sum_k sum_i f c_i),
 *   E_kin = sum 1/2 rho |u|^2, max |u|, count of nodes with a non-finite population,
 *   min rho_r, min rho_b -- over fluid nodes, reduced in FP64 in a fixed order.
 * totals != NULL synchronises the stream and returns LBM_EUNSTABLE when the blow-up check
 * trips (a non-finite population, a density below -1e-2 times the larger bulk density, or
 * max|u| > umax_unstable), also when a
 * periodic in-step check (diag_every) tripped earlier. */
lbm_status lbm_moments(lbm_ctx* ctx, double* rho_r, double* rho_b, double* u, double* pops,
                       double* totals);

/* Release the host-side context.  NULL-safe.  Does not free the caller's workspace. */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Static description of a status code. */
const char* lbm_status_string(lbm_status s);

/* Tiling of the fused step kernel: a block owns tiles of tx * ty node columns (tx * ty <=
 * 256 and a multiple of 32, or one of the 512-node tiles below) and marches them through z
 * in z-chunks; work units are (z-chunk, column) pairs taken chunk-major.  tz > 0:
 * ceil(nz / tz) chunks of near-equal length, one block per unit (tz must be 1 for D2Q9).
 * tz = 0: a persistent grid of as many blocks as fit on the device looping over the units,
 * with a chunk count chosen from that block count.  Default 32 x 8 x 16.
 * D3Q19 lattices in FP32/FP16/BF16 with nx % 32 == 0 and ny % 8 == 0 run the TMA-staged
 * kernel when tx x ty is 32 x 8 (for nx <= 256 as clusters of nx / 32 blocks that exchange
 * the x-halo in distributed shared memory; the cluster kernel also takes 32 x 4, with two
 * blocks per SM, and 64 x 4 when nx % 64 == 0, in clusters of nx / 64), the generic kernel
 * otherwise.  The ring kernel (the next plane's node state carried in registers, halo
 * columns as asynchronous remote stores) takes the CG and SC-multiphase models without
 * walls or the repulsion force: 32 x 16 and 64 x 8 tiles (one 512-thread block per SM;
 * D3Q19 only; where it does not apply, the step runs 32 x 8 tiles), and 64 x 4 tiles
 * where two of its blocks fit an SM (SC multiphase, or 16-bit storage), in clusters of
 * nx / tx <= 8 blocks; it gives the cluster kernel's results bit for bit.  Results are
 * bitwise independent of the shape within each kernel; the kernels agree to a few ulps of
 * the stored populations (the compiler fuses multiply-adds differently).  LBM_EINVAL for
 * shapes outside those limits. */
lbm_status lbm_set_tiling(lbm_ctx* ctx, int32_t tx, int32_t ty, int32_t tz);

/* ---- Batched stepping -------------------------------------------------------------
 * Many lattices (each an lbm_ctx) advance together: one persistent kernel launch per step
 * walks a device job table of all their work units (32 x 8 node columns times z-chunks
 * of <= tz planes, tz the job's lbm_set_tiling value, 16 when it is 0), so small lattices
 * do not pay one launch each and fill the GPU
 * together.  The per-node arithmetic is the generic step kernel's, so a lattice's result
 * is bitwise the same alone or in any mix (it may differ by a few ulps from a lattice
 * stepped with lbm_step_* on the TMA-staged kernel).  Jobs may have walls (halfway
 * bounce-back on their wall mask).  Jobs must be initialised, without the repulsion
 * force, with two-buffer streaming (LBM_STREAM_AB), of
 * the batch's storage precision and on the batch's stream, with K * Q * N < 2^31 (the
 * batched kernel indexes in 32 bits).  The periodic diagnostics (diag_every) do not run inside a batch; call
 * lbm_moments per job.
 *
 * lbm_batch_create: precision LBM_FP32, LBM_FP16 or LBM_BF16; capacity max_jobs lattices
 * and max_units work units.  ws == NULL: *ws_bytes receives the device workspace size
 * (caller-owned, 256-byte aligned, kept until lbm_batch_destroy).  LBM_EINVAL for another
 * precision or a non-positive capacity.
 * lbm_batch_units: work units a lattice occupies (for capacity and admission planning).
 * lbm_batch_set: the job list; job j takes nsteps[j] further steps over later
 * lbm_batch_step calls.  Uploads the table on the stream.  LBM_EINVAL when a job does not
 * fit the rules above or the capacity is exceeded, LBM_ESTATE for an uninitialised or
 * failed context.
 * lbm_batch_step: advances every job by min(nsteps, its remaining steps); use_graph != 0
 * replays the nsteps launches as one CUDA graph (built on the first call with that nsteps,
 * then reused; the table address is fixed, so lbm_batch_set does not invalidate it).
 * Asynchronous on the stream; updates each context's step count and current buffer.
 * lbm_batch_launch_count: step-kernel launches enqueued so far (graph nodes included).
 * lbm_batch_destroy: NULL-safe; does not touch the jobs or the workspace. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(int32_t precision, int32_t max_jobs, int32_t max_units, void* ws, size_t* ws_bytes,
                            void* stream, lbm_batch** out);
lbm_status lbm_batch_units(const lbm_ctx* ctx, int32_t* units);
lbm_status lbm_batch_set(lbm_batch* batch, lbm_ctx* const* jobs, const int32_t* nsteps, int32_t njobs);
lbm_status lbm_batch_step(lbm_batch* batch, int32_t nsteps, int32_t use_graph);
uint64_t lbm_batch_launch_count(const lbm_batch* batch);
lbm_status lbm_batch_destroy(lbm_batch* batch);

/* Number of kernel launches this context has enqueued since creation (for accounting). */
uint64_t lbm_launch_count(const lbm_ctx* ctx);

/* Exact checkpoint of the raw device state (stored deviations and reference densities),
 * for bitwise resume on the same precision and lattice; lbm_moments' canonical populations
 * are the portable FP64 form.  lbm_state_bytes: size of that state (0 for NULL).
 * lbm_save_state copies it to dst (host or device, caller-owned, lbm_state_bytes large),
 * synchronously; returns LBM_EUNSTABLE (state still written) if the blow-up check had
 * tripped.  The state is always written in the two-buffer layout (slot i of node x holds
 * direction i), also from an in-place context after an odd number of steps, so it loads
 * into a context of either streaming mode.  lbm_load_state restores it (solid: the wall mask as for lbm_init_fields, or
 * NULL), synchronously, and resets the step counter and blow-up status. */
size_t lbm_state_bytes(const lbm_ctx* ctx);
lbm_status lbm_save_state(lbm_ctx* ctx, void* dst);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* src, const uint8_t* solid);

/* Raw state of a range of z-planes, for domain decomposition (the halo planes of a z-slab
 * sub-domain; Sec. 2.3 notes that a single layer of boundary nodes shared between processes
 * suffices for the repulsion method).  The packed layout is that of lbm_save_state
 * restricted to the planes [z0, z0 + nplanes): for each of the K*Q population arrays, then
 * each of the K reference-density arrays, nplanes * nx * ny values of the storage type
 * (reference densities FP64 for FP64 storage, FP32 otherwise), x fastest.
 * lbm_state_planes_bytes: the packed size (0 for a NULL context or nplanes < 1).
 * lbm_get_state_planes copies the planes of the state the next step reads into buf,
 * lbm_set_state_planes writes buf into them; buf is host (pinned or pageable) or device
 * memory owned by the caller; both are enqueued on the context's stream and return at once
 * (pageable host memory makes the copy synchronous, as cudaMemcpyAsync does).  A state
 * frozen by a tripped blow-up check is not tracked here (read lbm_moments' status).
 * Errors: LBM_EINVAL for a NULL argument, z0 < 0, nplanes < 1 or z0 + nplanes > nz;
 * LBM_ESTATE before lbm_init_fields or with in-place streaming (LBM_STREAM_AA);
 * LBM_ECUDA on a CUDA error. */
size_t lbm_state_planes_bytes(const lbm_ctx* ctx, int32_t nplanes);
lbm_status lbm_get_state_planes(lbm_ctx* ctx, int32_t z0, int32_t nplanes, void* buf);
lbm_status lbm_set_state_planes(lbm_ctx* ctx, int32_t z0, int32_t nplanes, const void* buf);

/* Allocation-free totals (the paper has no counterpart; this serves callers that cannot
 * call cudaMalloc, e.g. a plugin whose host application's caching allocator has reserved
 * the device memory, or a loop that must never enter the driver's allocation path).
 * Computes the LBM_NTOTALS totals lbm_moments reports (same definitions, FP64, fixed-order
 * reduction) from caller-owned canonical populations, without a context or workspace.
 *   p      : lattice, model, nx/ny/nz and the force parameters (G, rho0_psi, body_force,
 *            rho_r0/rho_b0, umax_unstable) of the state; precision is ignored.
 *   pops   : DEVICE pointer, FP64 canonical populations [K][Q][N] (as lbm_moments exports).
 *   solid  : DEVICE pointer to the uint8 wall mask [N], or NULL.
 *   totals : host or device pointer to LBM_NTOTALS doubles (written).
 *   stream : cudaStream_t the work is enqueued on; the call synchronises it.
 * Scratch lives in one static __device__ array per device that loads the library, held
 * until process exit: 2 * LBM_NOALLOC_MAX_NODES FP64 densities (16 MiB), 1184 blocks x
 * LBM_NTOTALS FP64 partial sums (94,720 bytes) and a 256-byte result record, 16,872,192
 * bytes in all; nothing is allocated by the call.  The first call
 * on a device looks up that array's address (cudaGetSymbolAddress, with the caller's
 * device current) and so should come before any stream capture on that device.  Calls
 * share the array: calls that overlap on the GPU race and must be serialised.
 * The totals agree with lbm_moments' to rounding of the FP64 sums (about 1e-12 relative
 * on masses, E_kin, max|u| and minimum densities; momentum to 1e-13 of the mass): both sum
 * momentum as opposite-pair differences, but from different inputs (canonical FP64
 * populations here, the stored deviations there).
 * Not supported: the multirange SC model (LBM_MODEL_SC_MR) and CG with the repulsion force
 * (rep_pi != 0), whose force enters u and E_kin; both give LBM_EINVAL.
 * Errors: LBM_EINVAL for NULL pops or totals, pops or solid not in the memory of the current
 * device (host memory, or device memory of another GPU; managed memory is accepted),
 * N > LBM_NOALLOC_MAX_NODES, bad sizes or an unsupported model; LBM_ECUDA on a CUDA error;
 * LBM_EUNSTABLE when the blow-up check trips (totals written).  The call cannot know the
 * sizes of pops and solid: they must hold K*Q*N doubles and N bytes. */
enum { LBM_NOALLOC_MAX_NODES = 1 << 20 };
lbm_status lbm_totals_noalloc(const lbm_params* p, const double* pops, const uint8_t* solid, double* totals,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
