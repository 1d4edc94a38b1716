/*
 * tnmc.h - C ABI of the GB300 TNMCMC-1 slice-update library.
 *
 * The library implements the hot path of Tensor Network Markov Chain Monte
 * Carlo (TNMCMC-1, Algorithm 2 and SM II.A of arXiv 2509.23945): a 2D slice of
 * a 3D lattice is resampled with its two neighbouring slices held fixed as a
 * site-dependent field. The slice network is contracted row by row with a
 * boundary MPS of bond dimension chi (SM I.B), a candidate slice is drawn
 * spin by spin from the conditionals of that contraction (SM I.C), and the
 * candidate is accepted with the Metropolis-Hastings probability of Eq. (1)
 * using the exact energy difference.
 *
 * Conventions for every entry point:
 *  - Spins are int8 state indices v in [0, d) laid out [Lz][Ly][Lx] per chain
 *    (x fastest). For Ising d = 2 and index 0 is spin +1, index 1 is spin -1
 *    (the basis-vector convention of SM I.C). Potts uses d = q.
 *  - Couplings are int32 fixed point in units of 2^-20, layout
 *    [n_inst][3][Lz][Ly][Lx]; J[a][z][y][x] is the bond from (x, y, z) to its
 *    neighbour one step along axis a (0 = x, 1 = y, 2 = z), wrapping. On an
 *    open axis the wrapping bond must be 0. E = -sum_bonds J e(s_i, s_j) with
 *    e = s_i s_j (Ising) or delta(s_i, s_j) (Potts).
 *  - Device pointers are CUDA device addresses on the context's device; host
 *    pointers are ordinary host memory. Every call is ordered on the stream
 *    given to tnmc_create. The library never frees caller buffers.
 *  - Errors are returned as tnmc_status; tnmc_last_error() gives a message.
 *    A kernel that meets a non-finite conditional distribution or a
 *    non-finite Metropolis log-ratio latches TNMC_ERR_NONFINITE in a device
 *    status word of the context. Such a site is drawn from the uniform
 *    fallback (q stays a normalised distribution, so the chain stays exact)
 *    and a non-finite ratio rejects the move. The next synchronising call
 *    (tnmc_sync, tnmc_get_spins, tnmc_slice_logz) returns the latched status
 *    once and clears it. The tcgen05 GEMM engines (tnmc_set_tuning,
 *    tnmc_cta_gemm) bound their wait for the tensor cores; a wait that
 *    expires latches TNMC_ERR_TIMEOUT the same way (the CTA skips the rest of
 *    that GEMM and frees its tensor memory).
 *  - There is no CPU fallback: without a CUDA device tnmc_create fails.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef TNMC_H
#define TNMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnmc_ctx tnmc_ctx;

typedef enum {
  TNMC_OK = 0,
  TNMC_ERR_ARG = 1,        /* invalid argument (sizes, enums, null pointers)               */
  TNMC_ERR_ADJACENT = 2,   /* a batch holds two neighbouring slices of one chain: they do
                              not form a Markov blanket of each other (SM II.A)            */
  TNMC_ERR_OOM = 3,        /* device allocation failed                                     */
  TNMC_ERR_CUDA = 4,       /* a CUDA runtime call failed                                   */
  TNMC_ERR_TIMEOUT = 5,    /* a bounded device-side wait for the tensor cores expired      */
  TNMC_ERR_NONFINITE = 6,  /* a conditional or Metropolis ratio was not finite (latched)   */
  TNMC_ERR_STATE = 7       /* call not valid in the context's current state                */
} tnmc_status;

enum { TNMC_MODEL_EA_PM = 0, TNMC_MODEL_EA_GAUSS = 1, TNMC_MODEL_POTTS = 2 };

/* Arithmetic of the environment pass. F64: everything in double (CUDA
 * cores). F32: contractions, LQ factorisations and the one-sided Jacobi SVD
 * in float on the CUDA cores (tnmc_set_tuning can move the contractions to
 * 3xTF32 tensor-core products). BF16: the contractions with BF16 operands and
 * FP32 accumulation on the tensor cores, the factorisations as F32. In every
 * mode the conditionals are normalised in double, log q and the Metropolis
 * log-ratio are double and dE is an exact integer, so the chain stays exact;
 * precision moves only the acceptance rate. */
enum { TNMC_PREC_F64 = 0, TNMC_PREC_F32 = 1, TNMC_PREC_BF16 = 2 };

/* Which spins of a periodic slice are held fixed (the Potts experiments of
 * the main text fix "the spins on a randomly chosen line"):
 * R1 fixes one random row, so rows stay periodic rings;
 * R2 also fixes one random column, leaving an open rectangle. */
enum { TNMC_FIX_R1 = 0, TNMC_FIX_R2 = 1 };

enum { TNMC_PROPOSAL_TN = 0, TNMC_PROPOSAL_NET = 1, TNMC_PROPOSAL_CACHE = 2 };

/* One lattice geometry and the chains that live on it. */
typedef struct {
  int Lx, Ly, Lz;          /* extents, each >= 2                                      */
  int bc[3];               /* per axis: 1 periodic, 0 open (free)                       */
  int model;               /* TNMC_MODEL_*                                             */
  int q;                   /* Potts states (2..4); ignored for Ising models            */
  int chi;                 /* boundary-MPS bond dimension, 1..64                       */
  int precision;           /* TNMC_PREC_*; must be equal in every group of a context   */
  int fix_mode;            /* TNMC_FIX_*                                               */
  int n_chains;            /* chains on this lattice                                   */
  const double* betas;     /* host [n_chains] inverse temperatures, finite and >= 0      */
  const int32_t* instance_of_chain; /* host [n_chains], each in [0, n_inst)            */
  int n_inst;              /* disorder instances                                       */
  const int32_t* couplings;/* [n_inst][3][Lz][Ly][Lx] fixed point 2^-20                */
  int couplings_on_device; /* 1: couplings is a device pointer; 0: host pointer         */
  int layers;              /* 0 or 1: TNMCMC-1 slice updates; 2: TNMCMC-2 (see below)   */
} tnmc_config;

/* TNMCMC-2 (SM II.B, "coarse-graining with superspins"): with layers = 2 a
 * group's updates act on composite layers. Composite k normal to axis a joins
 * layers k and k + 1 (mod the extent); each site is a superspin with state
 * v = s_k + 2 s_k+1 of the two spin state indices (d = 4; Ising models only).
 * The couplings inside both layers and between them enter the tensors of the
 * 2D network; layers k - 1 and k + 2 are the held Markov blanket. The fixed
 * line / column of a periodic plane is a whole line of superspins. Every draw
 * of a composite update uses the Philox axis word axis | 16 (so it never
 * coincides with a TNMCMC-1 draw). In tnmc_slice_update the slice ids are the
 * composites' first layers (k + 1 inside the lattice on an open axis; two
 * composites of one chain at least 3 layers apart), new_spins_out holds
 * superspin states, and dE covers every bond of both layers. tnmc_sweep: sweep
 * t uses axis t mod 3 and composites starting at layers o, o + 2, ... with
 * o = (t / 3) mod 2, coloured like TNMCMC-1 slices (composites form a ring on
 * a periodic axis of even extent, else a path). The learned proposal is not
 * available for such groups (tnmc_net_init returns TNMC_ERR_ARG). */

/* Create a context holding n_groups lattices (uneven sizes allowed) and their
 * chains, all updated together by tnmc_sweep. Copies betas, instances and
 * couplings to the device; spins start at index 0 (call tnmc_set_spins).
 * cuda_stream: a cudaStream_t or NULL for the legacy default stream.
 * Errors: TNMC_ERR_ARG, TNMC_ERR_OOM, TNMC_ERR_CUDA (no device). */
tnmc_status tnmc_create(tnmc_ctx** out, const tnmc_config* cfgs, int n_groups, void* cuda_stream);

/* Copy spins of one group in or out: [n_chains][Lz][Ly][Lx] int8.
 * on_device selects whether the pointer is a device (1) or host (0) address.
 * tnmc_get_spins synchronises the stream and returns latched kernel errors. */
tnmc_status tnmc_set_spins(tnmc_ctx* ctx, int group, const int8_t* spins, int on_device);
tnmc_status tnmc_get_spins(tnmc_ctx* ctx, int group, int8_t* out, int on_device);

/* One TNMCMC-1 slice update of n_items (chain, slice) pairs of one group, all
 * normal to `axis`, run in one launch (Algorithm 2, SampleLayer + MH).
 * chain_ids, slice_ids: host [n_items]; slices of the same chain must be
 * pairwise non-adjacent (else TNMC_ERR_ADJACENT).
 * The random draws use Philox4x32-10 with key = seed and counter
 * (purpose << 24 | index, slice | axis << 16, step, global chain id).
 * proposal: TNMC_PROPOSAL_TN, or TNMC_PROPOSAL_NET once a network is loaded.
 * Outputs are device arrays [n_items] (new_spins_out: [n_items][Lmax*Lmax],
 * the active region row-major with row stride Lmax = max in-plane extent);
 * each may be NULL. dE is in units of 2^-20. If write_back is 0 the lattice
 * is left unchanged (proposal evaluation only). */
tnmc_status tnmc_slice_update(tnmc_ctx* ctx, int group, int axis, int n_items,
                              const int32_t* chain_ids, const int32_t* slice_ids,
                              uint64_t seed, uint64_t step, int proposal, int write_back,
                              int8_t* new_spins_out, double* logq_new, double* logq_old,
                              uint8_t* accept, int64_t* dE);

/* n_sweeps sweeps of every chain of every group: sweep t uses axis t mod 3 and
 * updates the colour classes of that axis in turn (two for even or open
 * axes, three for odd periodic ones), all chains and groups of a class in
 * one launch. The sweep counter t is kept by the context (tnmc_get_sweep).
 * With use_graph = 1 the three axis sweeps are captured once as CUDA graphs
 * and replayed. accept_out: device [total chains] uint32 counters that are
 * incremented per accepted slice (may be NULL). */
tnmc_status tnmc_sweep(tnmc_ctx* ctx, int n_sweeps, uint64_t seed, int use_graph, uint32_t* accept_out);
tnmc_status tnmc_get_sweep(tnmc_ctx* ctx, uint64_t* t);
tnmc_status tnmc_set_sweep(tnmc_ctx* ctx, uint64_t t);

/* Per-chain observables of one group into device out [n_chains][3]:
 * energy per site E/N, magnetisation per site M = mean of s (Ising values; for
 * Potts the order parameter (q max_a n_a / N - 1)/(q - 1)), and the overlap
 * q = (1/N) sum_i s_i s_i' with chain partner[c] (host [n_chains], or NULL
 * for chain c ^ 1). The overlap is the spin-glass order parameter of the main
 * text ("Sampling 3D spin glasses"). */
tnmc_status tnmc_observables(tnmc_ctx* ctx, int group, const int32_t* partner, double* out);

/* Test hook: log Z of the slice network of (chain, axis, slice) with the same
 * fixed line that tnmc_slice_update draws for (seed, step), contracted at the
 * context's chi. Exact when chi reaches the exact bond dimension. Host output. */
tnmc_status tnmc_slice_logz(tnmc_ctx* ctx, int group, int chain, int axis, int slice,
                            uint64_t seed, uint64_t step, double* logz);

/* Kernel configuration of a context (chosen by the autotuner in
 * paper_2509_23945_gb300/autotune.py, or left at the defaults):
 *   gemm_mode     engine of the contractions, a TNMC_GEMM_* value: F32 takes
 *                 FFMA (default), MMA_TF32X3 or UMMA_TF32X3; BF16 takes
 *                 MMA_BF16 (default) or UMMA_BF16; ignored for F64; any other
 *                 value is TNMC_ERR_ARG. The UMMA engines run tcgen05.mma on
 *                 the LQ route's contractions with operands staged in
 *                 24 KB of dynamic shared memory (reserved whatever eig_smem
 *                 says); the density-matrix route runs the mma.sync engine
 *                 of the same rounding instead. They are compiled into a
 *                 kernel instance of their own, which runs one CTA per SM.
 *   eig_smem      1: keep the factorisations' working matrices (one-sided
 *                 Jacobi rows, LQ panels; the eigenproblem of route 1) in
 *                 shared memory when they fit
 *   jac_floor     convergence floor of the route-1 eigensolver: 0 none,
 *                 1 eps^2 n max|a_ii|, 2 eps max|a_ii|
 *   ctas_per_sm   1 or 2 resident slice CTAs per SM asked for; the kernel
 *                 instance's occupancy caps it (tnmc_get_tuning reports the
 *                 value in use; the tcgen05 instance runs one), and the
 *                 request stands across later changes of the other fields
 *   route         truncation (SM I.B): 0 (default) the canonical SVD cut,
 *                 right-canonicalised by Householder LQ with each bond cut by
 *                 LQ + one-sided Jacobi SVD; 1 the same cut from the
 *                 eigenvectors of the reduced density matrix, which squares
 *                 singular values and so resolves a kept direction only to
 *                 sqrt(eps) of the largest (opt-in, for comparison)
 *   gemm_tile     output tile of the CUDA-core (FFMA) GEMMs of F32 and BF16
 *                 contexts (the LQ trailing updates run them in every
 *                 engine): 0 (default) 64 x 64, 1 32 x 32, 2 128 x 64;
 *                 each tile is its own compiled kernel. F64 contexts take 0.
 * gemm_mode and route 1 change the arithmetic, so they change results;
 * eig_smem, ctas_per_sm and gemm_tile do not (every output element of a
 * GEMM sums its products in the same order whatever the tile).
 * Any field set to -1 keeps its current value. Graphs are re-captured after a change. */
typedef struct {
  int gemm_mode;
  int eig_smem;
  int jac_floor;
  int ctas_per_sm;
  int route;
  int gemm_tile;
} tnmc_tuning;
tnmc_status tnmc_set_tuning(tnmc_ctx* ctx, const tnmc_tuning* t);
tnmc_status tnmc_get_tuning(tnmc_ctx* ctx, tnmc_tuning* t);

/* Test hook: scale every slice weight's inverse temperature by `factor` when
 * building proposals (the Metropolis step keeps the true beta). 1.0 = normal.
 * factor must be > 0; +inf is accepted and makes every proposal weight
 * non-finite, which the status word reports (a host-made failure for tests). */
tnmc_status tnmc_set_proposal_beta_factor(tnmc_ctx* ctx, double factor);

/* Tensor-network proposals drawn from one environment build (main text: "draw
 * a batch of candidate samples ... accept one"; the environments E_r depend
 * only on the held spins, SM II.A). n_prop = 1 (default) is Algorithm 2. With
 * n_prop = K > 1 every slice update builds its environments once and runs K
 * Metropolis-Hastings steps of an independence sampler on the slice: proposal
 * j is drawn from the same q and accepted against the current slice with
 * Eq. (1) (exact for any K). Proposal 0 draws as the single update does;
 * proposals j >= 1 use Philox purposes 5 (site draws, index (j-1) * active
 * sites + site) and 6 (Metropolis draw, index j-1). tnmc_slice_update then
 * reports log q of the original (logq_old) and final (logq_new) slice, the
 * number of accepted proposals (accept) and E(final) - E(original) (dE);
 * accept_out of tnmc_sweep counts accepted proposals; the replay buffer of the
 * learned proposal records single-proposal updates only. n_prop in 1..64. */
tnmc_status tnmc_set_proposals_per_env(tnmc_ctx* ctx, int n_prop);

/* n_sweeps sweeps of single-spin Metropolis on every chain (the method the
 * paper compares TNMCMC with; main text, "Sampling 3D spin glasses"; SM III):
 * a spin flips with probability min(1, exp(-beta dE)), dE = 2 s_i h_i, in two
 * checkerboard half-sweeps per sweep (colour (x + y + z) mod 2). The uniform
 * of site i = (z Ly + y) Lx + x in half-sweep c of Metropolis sweep t is
 * Philox purpose 7, index i, slice c, axis 0, step t, global chain id; t
 * counts this context's Metropolis sweeps from 0. Ising models only, on
 * bipartite lattices (every periodic extent even), else TNMC_ERR_ARG.
 * accept_out: device [total chains] uint32 flip counters or NULL. */
tnmc_status tnmc_metropolis_sweep(tnmc_ctx* ctx, int n_sweeps, uint64_t seed, uint32_t* accept_out);

/* Cache of environments built for earlier held fields (the Conclusions:
 * slices are resampled under fields from their held neighbours, so
 * contractions are frequent; keeping environments of "typical" fields makes
 * them needed only occasionally, at some cost in acceptance).
 * tnmc_cache_build contracts, for every chain, axis and slice of the context,
 * the environment stack E_1..E_m (SM I.B) of the current held spins, with the
 * fixed line / column drawn as tnmc_slice_update draws them for (seed, step),
 * into a cache slot in device memory (allocated by the first call; it holds
 * chains x 3 x max extent slots of one environment stack each; TNMC_ERR_OOM
 * if that does not fit). A later build overwrites every slot. TNMCMC-1 groups
 * only (TNMC_ERR_ARG with composite layers).
 * A cached update uses its slot's fixed lines and environments with the row
 * weights of the current held spins, then draws, evaluates log q of the
 * current slice and applies Eq. (1) with the exact dE as usual (the draws of
 * the single update of the same slice, step and chain). The proposal depends
 * on the held spins and the cache, not on the slice itself, so the chain is
 * exact while the cache is unchanged; rebuilding the cache from a chain's own
 * later state makes the proposal depend on the chain's past, and exactness
 * then holds between rebuilds only.
 * tnmc_slice_update with proposal TNMC_PROPOSAL_CACHE proposes every item
 * from the cache (TNMC_ERR_STATE before a build). tnmc_set_cache_mix(on = 1,
 * fresh_every = k) makes tnmc_sweep propose from the cache except on sweeps t
 * with k > 0 and t mod k = k - 1, which contract afresh (k = 0: always the
 * cache); on = 0 turns the cache off for sweeps (the default). Sweeps that
 * propose with the learned network (tnmc_set_proposal_mix) do not use the
 * cache. The cache is not part of a checkpoint. The paper has no
 * implementation of this cache. */
tnmc_status tnmc_cache_build(tnmc_ctx* ctx, uint64_t seed, uint64_t step);
tnmc_status tnmc_set_cache_mix(tnmc_ctx* ctx, int on, int fresh_every);

/* Wait for the stream and return any latched device-side error. */
tnmc_status tnmc_sync(tnmc_ctx* ctx);

/* Number of sites so far whose conditional fell back to the uniform
 * distribution (empty or non-finite truncated conditionals), host output. */
tnmc_status tnmc_events(tnmc_ctx* ctx, uint64_t* count);

/* Device bytes held by the context (workspace, environments, lattices). */
tnmc_status tnmc_memory(tnmc_ctx* ctx, size_t* bytes);

/* Checkpoint to / from a file: spins of every group and the sweep counter;
 * with a learned proposal also its weights, the Adam moments and step count,
 * the replay buffer (contents and fill counter) and the proposal schedule.
 * Loading a checkpoint that holds a network needs a context on which
 * tnmc_net_init was called with the same channels, layers and buffer slots
 * (else TNMC_ERR_STATE). A resumed run is bitwise identical to an
 * uninterrupted one because every draw is counter based. Both calls
 * synchronise the context's stream. Errors: TNMC_ERR_ARG (file cannot be
 * opened, not a checkpoint of this context, truncated), TNMC_ERR_STATE,
 * TNMC_ERR_CUDA. */
tnmc_status tnmc_save(tnmc_ctx* ctx, const char* path);
tnmc_status tnmc_load(tnmc_ctx* ctx, const char* path);

/* ---------------------------------------------------------------------------
 * Learned slice proposal. The paper has no learned proposal; its Conclusions
 * only suggest replacing frequent contractions by cached knowledge of typical
 * fields. This network is an independence proposal inside the same exact
 * Metropolis-Hastings step (Eq. (1)), so any positive q keeps the chain exact.
 * A masked-convolution autoregressive network (PixelCNN masks) over the active
 * region in the sampler's raster order: layer 0 maps the spin one-hot (mask A)
 * plus a 3x3 convolution of the conditioning features (log phi(v) of the held
 * field and beta*J of the four in-plane bonds) to `channels` maps with ReLU;
 * layers 1..layers-2 add a ReLU residual (mask B); the last layer gives d
 * logits per site. Parameters are FP32, laid out per layer as
 * ws[cout][cin][3][3], wc[cout][d+4][3][3], b[cout]. */

/* Allocate and initialise the network (uniform He initialisation from Philox
 * draws with `seed`) and a replay buffer of buffer_slots accepted slices.
 * All groups must share d. Errors: TNMC_ERR_ARG, TNMC_ERR_STATE (already
 * initialised), TNMC_ERR_OOM. */
tnmc_status tnmc_net_init(tnmc_ctx* ctx, int channels, int layers, uint64_t seed, int buffer_slots);
tnmc_status tnmc_net_param_count(tnmc_ctx* ctx, size_t* n);
/* Copy all parameters in or out ([n_params] float, device or host pointer). */
tnmc_status tnmc_net_set_params(tnmc_ctx* ctx, const float* w, int on_device);
tnmc_status tnmc_net_get_params(tnmc_ctx* ctx, float* w, int on_device);

/* Proposal schedule of tnmc_sweep: net_every = 0 uses the tensor network only;
 * net_every = k uses the network on sweeps t with t mod k = k - 1 (k = 2
 * alternates 1:1). record = 1 stores accepted tensor-network slices
 * (conditioning features and spins) in the replay buffer: item i of a
 * recording launch owns slot (positions offered before the launch + i) mod
 * slots, so the buffer's contents are reproducible; a rejected item leaves its
 * slot as it was. */
tnmc_status tnmc_set_proposal_mix(tnmc_ctx* ctx, int net_every, int record);
/* Recording positions offered to the replay buffer so far (it wraps around). */
tnmc_status tnmc_net_buffer_count(tnmc_ctx* ctx, uint64_t* count);

/* n_steps Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the mean over a
 * batch of replay slices of -log q(s) / (active sites). Batches are Philox
 * draws among the filled slots. losses: host [n_steps] or NULL. Gradients are
 * summed over slices in a fixed order (bitwise reproducible).
 * Errors: TNMC_ERR_STATE without a network or with an empty buffer. */
tnmc_status tnmc_net_train(tnmc_ctx* ctx, int n_steps, int batch, float lr, uint64_t seed, double* losses);

/* One Adam step (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected, the same update tnmc_net_train applies) with a caller-given
 * gradient grad[n_params] (device or host pointer), learning rate lr >= 0.
 * Advances the context's Adam step count. Synchronous. For custom training
 * loops and for checking the optimiser against a reference. */
tnmc_status tnmc_net_adam_step(tnmc_ctx* ctx, const float* grad, int on_device, float lr);

/* Test hook: teacher-forced pass of the network on the current spins of
 * n_items slices (same geometry draw as tnmc_slice_update for seed, step).
 * logits_out: device [n_items][d][Lmax*Lmax] or NULL; logq_out: device
 * [n_items] or NULL; grad_out: device [n_params] gradient of the mean over the
 * items of -log q / (active sites), or NULL. */
tnmc_status tnmc_net_eval(tnmc_ctx* ctx, int group, int axis, int n_items, const int32_t* chain_ids,
                          const int32_t* slice_ids, uint64_t seed, uint64_t step, float* logits_out,
                          double* logq_out, float* grad_out);

/* Allocation-free variant of tnmc_slice_logz, for callers that cannot allocate
 * device memory: plugins hosted by frameworks that own the whole device memory
 * pool, or services that allocate once at start-up and may not call cudaMalloc
 * later. The paper has no counterpart; it is a packaging of the log Z hook.
 * No context is needed and nothing is allocated: the kernel's scratch is a
 * fixed 2 MiB device array inside this library, and a small header array
 * holds the call's lattice descriptor; both are reserved on every GPU that
 * loads the library until the process exits.
 * Inputs: spins (device, int8 [Lz][Ly][Lx]) and couplings (device, int32
 * [3][Lz][Ly][Lx], units 2^-20) of one chain; bc[3] (host); Ising models only
 * (TNMC_MODEL_EA_PM or TNMC_MODEL_EA_GAUSS); extents 2..16; chi 1..16;
 * beta finite and >= 0; FP64 arithmetic. The fixed line is drawn from
 * (seed, step) as in tnmc_slice_update with global chain id 0. Output:
 * *logz_out (device double). Work is queued on cuda_stream (NULL: legacy
 * default stream); the caller synchronises. The first call on a device, with
 * that device current, resolves the scratch address once. All calls share the
 * scratch and the header arrays: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller. Every value the
 * kernel reads from the scratch is written earlier in the same call, so
 * nothing needs clearing between calls.
 * Errors: TNMC_ERR_ARG for sizes beyond these limits or invalid arguments,
 * TNMC_ERR_CUDA if a launch fails. */
tnmc_status tnmc_slice_logz_noalloc(const int8_t* spins, const int32_t* couplings, int Lx, int Ly, int Lz,
                                    const int* bc, int model, double beta, int chi, int axis, int slice,
                                    uint64_t seed, uint64_t step, int fix_mode, double* logz_out,
                                    void* cuda_stream);

/* Measured peak of the arithmetic that bounds the slice kernel: the fused
 * multiply-add throughput of the current device's CUDA cores in FP32
 * (precision TNMC_PREC_F32) or FP64 (TNMC_PREC_F64), in flop/s (2 per FMA).
 * The paper has no counterpart; it is the roofline denominator of the
 * benchmark. A grid of 8 CTAs x 256 threads per SM runs 8 independent FMA
 * chains per thread; one untimed launch, then one launch timed with CUDA
 * events on cuda_stream (NULL: legacy default stream). Synchronous; allocates
 * nothing. Output: *flops_per_s (host). Errors: TNMC_ERR_ARG for another
 * precision or a NULL output, TNMC_ERR_CUDA if a launch fails. */
tnmc_status tnmc_probe_alu_peak(int precision, void* cuda_stream, double* flops_per_s);

/* GEMM engines of the slice kernel's contractions (SM I.B: every step of the
 * environment pass is a product of small dense matrices).
 *   FFMA:         FP32 fused multiply-adds on the CUDA cores.
 *   MMA_TF32X3:   warp-level mma.sync, each operand split into two TF32 parts,
 *                 three products per term, FP32 accumulation.
 *   MMA_BF16:     warp-level mma.sync, BF16 operands, FP32 accumulation.
 *   UMMA_TF32X3:  the TF32 split of MMA_TF32X3 issued as tcgen05.mma
 *                 (kind::tf32) with the accumulator in tensor memory.
 *   UMMA_BF16:    BF16 operands, tcgen05.mma (kind::f16), FP32 accumulator in
 *                 tensor memory. */
enum {
  TNMC_GEMM_FFMA = 0,
  TNMC_GEMM_MMA_TF32X3 = 1,
  TNMC_GEMM_MMA_BF16 = 2,
  TNMC_GEMM_UMMA_TF32X3 = 3,
  TNMC_GEMM_UMMA_BF16 = 4
};

/* One CTA-level GEMM per CTA, on its own: C_b = alpha op(A_b) op(B_b) +
 * beta C_b for b = 0 .. batch-1, with A_b = A + b strideA (elements), and so
 * on. All matrices are FP32, row-major, on the device: op(A) is M x K
 * (transA: A is stored K x M with leading dimension lda), op(B) is K x N
 * (transB: B is stored N x K), C is M x N with leading dimension ldc; beta ==
 * 0 never reads C. Each CTA runs the selected engine exactly as the slice
 * kernel does, so the engines can be checked against a host product and timed
 * at full occupancy. The paper has no counterpart. Work is queued on
 * cuda_stream (NULL: legacy default stream); the call synchronises it.
 * Allocates nothing. Errors: TNMC_ERR_ARG for an unknown engine, batch
 * outside 0..65535, negative sizes or strides, leading dimensions too small
 * or NULL matrices; TNMC_ERR_CUDA if a launch fails; TNMC_ERR_TIMEOUT if a
 * tensor-core engine's bounded wait for its MMAs expired (the CTA then skips
 * its remaining tiles and frees its tensor memory). */
tnmc_status tnmc_cta_gemm(int engine, int batch, int M, int N, int K, float alpha, const float* A, int lda,
                          long long strideA, int transA, const float* B, int ldb, long long strideB, int transB,
                          float beta, float* C, int ldc, long long strideC, void* cuda_stream);

const char* tnmc_last_error(const tnmc_ctx* ctx);
void tnmc_destroy(tnmc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TNMC_H */
