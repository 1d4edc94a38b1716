// C ABI of the slice-update library (declared in include/tnmc.h).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tnmc.h"
#include "common.cuh"
#include "slice_launch.cuh"

using namespace tnmc;

void tnmc_launch_metropolis(const Group& g, uint64_t seed, uint32_t t, int colour, unsigned int* acc,
                            cudaStream_t stream);

struct GroupHost {
  tnmc_config cfg;
  int d;
  size_t vol;
  int chain_base;
  int8_t* d_spins = nullptr;
  int32_t* d_J = nullptr;
  double* d_beta = nullptr;
  int32_t* d_inst = nullptr;
};

struct tnmc_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;   // private stream on which sweeps are captured into graphs
  int device = 0;
  int precision = TNMC_PREC_F64;
  std::vector<GroupHost> groups;
  Group* d_groups = nullptr;
  int total_chains = 0;
  WsLayout lay{};
  char* d_ws = nullptr;
  size_t ws_stride = 0;
  int max_ctas = 0;
  size_t dyn_smem = 0;
  int jac_floor = 0;
  int gemm_mode = GEMM_FFMA;
  int gemm_tile = 0;       // CUDA-core GEMM tile of the float kernel (0 64x64, 1 32x32, 2 128x64)
  int ctas_per_sm = 2;
  int req_ctas = 2;        // resident CTAs per SM asked for (tnmc_set_tuning); the kernel's occupancy caps it
  int alloc_ctas = 0;      // CTAs the workspace was sized for
  int sms = 0;
  size_t eig_bytes = 0;    // dynamic shared memory wanted by the density-matrix route
  size_t lq_bytes = 0;     // ... and by the LQ route
  int route = ROUTE_LQ;
  int n_prop = 1;          // tensor-network proposals per environment build
  uint64_t h_metro = 0;    // single-spin Metropolis sweeps done
  int smem_on = 1;         // tuning: factorisations in dynamic shared memory when they fit
  int fact_smem = 0;       // 1: the factorisations use the dynamic shared memory
  int umma_stage = 0;      // 1: the dynamic shared memory holds the tcgen05 GEMM staging
  unsigned long long* d_sweep = nullptr;
  unsigned long long* d_events = nullptr;
  unsigned int* d_status = nullptr;   // latched StatusBits
  unsigned long long h_sweep = 0;
  int* d_items = nullptr;  // [3][max_items]
  int max_items = 0;
  double* d_logz = nullptr;
  double env_beta_factor = 1.0;
  cudaGraphExec_t graphs[3] = {nullptr, nullptr, nullptr};
  uint64_t graph_seed[3] = {0, 0, 0};
  uint32_t* graph_acc[3] = {nullptr, nullptr, nullptr};
  size_t bytes = 0;
  std::string err;
  // learned proposal
  bool net_on = false;
  NetLayout net{};
  float* d_W = nullptr;
  float* d_m1 = nullptr;
  float* d_m2 = nullptr;
  int adam_t = 0;
  float* d_net_ws = nullptr;      // slice-kernel CTAs
  size_t net_ws_stride = 0;
  int Pmax = 0;
  float* d_train_ws = nullptr;    // training CTAs
  size_t train_ws_stride = 0;
  int train_ctas = 0;
  float* d_gbuf = nullptr;
  double* d_loss = nullptr;
  int* d_slots = nullptr;
  int max_batch = 0;
  float* d_rb_cond = nullptr;
  int8_t* d_rb_spins = nullptr;
  int* d_rb_meta = nullptr;
  unsigned long long* d_rb_count = nullptr;
  int rb_slots = 0;
  int net_every = 0;
  int record = 0;
  // cache of environments (tnmc_cache_build / tnmc_set_cache_mix)
  char* d_cache = nullptr;
  size_t cache_stride = 0, cache_dims_off = 0, cache_meta_off = 0;
  int cache_lmax = 0;
  int cache_ready = 0;
  int cache_on = 0;
  int cache_every = 0;
};

static tnmc_status fail(tnmc_ctx* c, tnmc_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CU(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return fail(ctx, TNMC_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

static void drop_graphs(tnmc_ctx* ctx) {
  for (auto& gexec : ctx->graphs)
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
}

// After a stream synchronisation: return (and clear) a status latched by a kernel.
static tnmc_status read_status(tnmc_ctx* ctx) {
  unsigned int v = 0;
  if (cudaMemcpy(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(ctx, TNMC_ERR_CUDA, "reading the device status word");
  if (!v) return TNMC_OK;
  cudaMemset(ctx->d_status, 0, sizeof(unsigned int));
  if (v & ST_TIMEOUT)
    return fail(ctx, TNMC_ERR_TIMEOUT,
                "a tensor-core GEMM's bounded wait for its MMAs expired (the CTA skipped the rest of that GEMM)");
  return fail(ctx, TNMC_ERR_NONFINITE,
              "a kernel met a non-finite conditional or Metropolis ratio (the move was rejected or drawn from the "
              "uniform fallback)");
}

static tnmc_status dalloc(tnmc_ctx* ctx, void** p, size_t n) {
  cudaError_t e = cudaMalloc(p, n ? n : 1);
  if (e != cudaSuccess) return fail(ctx, TNMC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  ctx->bytes += n;
  return TNMC_OK;
}

// Work positions of one colour-class launch of a sweep (the kernel's find_item): a group of
// composite layers takes the larger count of its two offsets, so one captured graph serves both.
static int items_for(const tnmc_ctx* ctx, int axis, int colour) {
  int n = 0;
  for (const auto& g : ctx->groups) {
    const int L[3] = {g.cfg.Lx, g.cfg.Ly, g.cfg.Lz};
    int per;
    if (g.cfg.layers == 2)
      per = std::max(composite_count(L[axis], g.cfg.bc[axis], 0, colour),
                     composite_count(L[axis], g.cfg.bc[axis], 1, colour));
    else
      per = colour_count(L[axis], g.cfg.bc[axis], colour);
    n += per * g.cfg.n_chains;
  }
  return n;
}

__global__ void bump_counter(unsigned long long* c, unsigned long long n) { *c += n; }

template <typename R>
static void launch_phase(tnmc_ctx* ctx, PhaseParams& P, int total) {
  P.ws = ctx->d_ws;
  P.ws_stride = ctx->ws_stride;
  P.lay = ctx->lay;
  P.groups = ctx->d_groups;
  P.n_groups = (int)ctx->groups.size();
  P.event_counter = ctx->d_events;
  P.status = ctx->d_status;
  P.env_beta_factor = ctx->env_beta_factor;
  P.eig_smem = ctx->fact_smem;
  P.umma_stage = ctx->umma_stage;
  P.dyn_bytes = ctx->dyn_smem;
  P.route = ctx->route;
  P.n_prop = ctx->n_prop;
  P.jac_floor = ctx->jac_floor;
  P.gemm_mode = ctx->gemm_mode;
  P.gemm_tile = ctx->precision == TNMC_PREC_F64 ? 0 : ctx->gemm_tile;
  P.cache = ctx->d_cache;
  P.cache_stride = ctx->cache_stride;
  P.cache_lmax = ctx->cache_lmax;
  P.cache_dims_off = ctx->cache_dims_off;
  P.cache_meta_off = ctx->cache_meta_off;
  if (!ctx->d_cache) P.cache_mode = CACHE_OFF;
  if (ctx->net_on) {
    P.net = ctx->net;
    P.net_W = ctx->d_W;
    P.net_ws = ctx->d_net_ws;
    P.net_ws_stride = ctx->net_ws_stride;
    P.net_Pmax = ctx->Pmax;
    P.rb_cond = ctx->d_rb_cond;
    P.rb_spins = ctx->d_rb_spins;
    P.rb_meta = ctx->d_rb_meta;
    P.rb_counter = ctx->d_rb_count;
    P.rb_slots = ctx->rb_slots;
  }
  int grid = total < ctx->max_ctas ? total : ctx->max_ctas;
  if (grid < 1) return;
  slice_launch<R>(P, total, grid, ctx->dyn_smem, ctx->stream);
  // the items of a recording launch own the next `total` replay positions
  if (P.record && P.rb_slots > 0) bump_counter<<<1, 1, 0, ctx->stream>>>(ctx->d_rb_count, (unsigned long long)total);
}

static void launch(tnmc_ctx* ctx, PhaseParams& P, int total) {
  if (ctx->precision == TNMC_PREC_F64) launch_phase<double>(ctx, P, total);
  else launch_phase<float>(ctx, P, total);   // FP32 and BF16 contractions both run the float kernel
}

__global__ void bump_sweep(unsigned long long* t) { *t += 1ull; }

constexpr size_t kDynSmemCap = 180 * 1024;

// Dynamic shared memory of the slice kernel for the context's route and tuning; returns the
// resident CTAs per SM that the occupancy calculator allows with it.
static bool umma_mode(int m) { return m == GEMM_UMMA_TF32X3 || m == GEMM_UMMA_BF16; }

// Kernel instance of a float context: the tcgen05 instance for the UMMA engines, else its GEMM tile.
static int float_instance(const tnmc_ctx* ctx) {
  return umma_mode(ctx->gemm_mode) ? kSliceInstanceUmma : ctx->gemm_tile;
}

static int apply_smem(tnmc_ctx* ctx) {
  size_t want = ctx->route == ROUTE_DM ? ctx->eig_bytes : ctx->lq_bytes;
  // the tcgen05 GEMM stages its operands in the same region, between factorisations (LQ route only),
  // whether or not the factorisations use it: the engine, not eig_smem, decides the arithmetic
  const size_t stage = (umma_mode(ctx->gemm_mode) && ctx->route != ROUTE_DM) ? (size_t)kUmmaStageBytes + 128 : 0;
  // room left for dynamic shared memory: the device's opt-in limit per block minus the kernel's static part
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  cudaFuncAttributes fa{};
  if (ctx->precision == TNMC_PREC_F64) slice_attributes<double>(&fa);
  else slice_attributes<float>(&fa, float_instance(ctx));
  const size_t room = (size_t)optin > fa.sharedSizeBytes + 1024 ? (size_t)optin - fa.sharedSizeBytes - 1024 : 0;
  const size_t cap = room < kDynSmemCap ? room : kDynSmemCap;
  if (ctx->route != ROUTE_DM && want > cap) want = cap;     // the LQ route uses what fits (panel, Jacobi rows)
  if (!ctx->smem_on || want > cap) want = 0;
  ctx->fact_smem = want > 0;
  if (stage > want && stage <= cap) want = stage;
  ctx->umma_stage = stage > 0 && want >= stage;
  if (want) {
    cudaError_t ea = ctx->precision == TNMC_PREC_F64
        ? slice_set_dyn_smem<double>((int)want)
        : slice_set_dyn_smem<float>((int)want, float_instance(ctx));
    if (ea != cudaSuccess) { want = 0; ctx->fact_smem = 0; ctx->umma_stage = 0; }
  }
  ctx->dyn_smem = want;
  int occ = 0;
  if (ctx->precision == TNMC_PREC_F64)
    slice_occupancy<double>(&occ, ctx->dyn_smem);
  else
    slice_occupancy<float>(&occ, ctx->dyn_smem, float_instance(ctx));
  return occ;
}

extern "C" {

tnmc_status tnmc_create(tnmc_ctx** out, const tnmc_config* cfgs, int n_groups, void* cuda_stream) {
  tnmc_ctx* ctx = nullptr;
  if (!out || !cfgs || n_groups < 1) return TNMC_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return TNMC_ERR_CUDA;
  ctx = new tnmc_ctx();
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&ctx->device);
  ctx->precision = cfgs[0].precision;
  int Mmax = 1, Lmax = 2, dmax = 2, chimax = 1;
  int base = 0;
  for (int gi = 0; gi < n_groups; ++gi) {
    const tnmc_config& c = cfgs[gi];
    const int L[3] = {c.Lx, c.Ly, c.Lz};
    auto bad = [&](const char* m) { delete ctx; return TNMC_ERR_ARG; };
    for (int a = 0; a < 3; ++a)
      if (L[a] < 2 || L[a] > 128 || (c.bc[a] != 0 && c.bc[a] != 1)) return bad("extent");
    if (c.model < 0 || c.model > 2) return bad("model");
    if (c.chi < 1 || c.chi > 64) return bad("chi");
    if (c.precision != ctx->precision ||
        (c.precision != TNMC_PREC_F64 && c.precision != TNMC_PREC_F32 && c.precision != TNMC_PREC_BF16))
      return bad("precision");
    if (c.fix_mode != TNMC_FIX_R1 && c.fix_mode != TNMC_FIX_R2) return bad("fix");
    if (c.n_chains < 1 || c.n_inst < 1 || !c.betas || !c.instance_of_chain || !c.couplings) return bad("chains");
    if (c.layers != 0 && c.layers != 1 && c.layers != 2) return bad("layers");
    // composite layers of Ising superspins (SM II.B): d = 2 x 2
    if (c.layers == 2 && c.model == TNMC_MODEL_POTTS) return bad("layers");
    const int d = c.layers == 2 ? 4 : (c.model == TNMC_MODEL_POTTS ? c.q : 2);
    if (d < 2 || d > 4) return bad("q");
    for (int i = 0; i < c.n_chains; ++i)
      if (c.instance_of_chain[i] < 0 || c.instance_of_chain[i] >= c.n_inst) return bad("instance");
    for (int i = 0; i < c.n_chains; ++i)
      if (!std::isfinite(c.betas[i]) || c.betas[i] < 0.0) return bad("beta");
    GroupHost g;
    g.cfg = c;
    g.cfg.layers = c.layers == 2 ? 2 : 1;
    g.d = d;
    g.vol = (size_t)L[0] * L[1] * L[2];
    g.chain_base = base;
    base += c.n_chains;
    ctx->groups.push_back(g);
    for (int a = 0; a < 3; ++a) {
      Mmax = std::max(Mmax, L[(a + 2) % 3]);
      Lmax = std::max(Lmax, L[(a + 1) % 3]);
    }
    Lmax = std::max(Lmax, Mmax);
    Mmax = Lmax;
    dmax = std::max(dmax, d);
    chimax = std::max(chimax, c.chi);
  }
  ctx->total_chains = base;
  tnmc_status st;
  std::vector<Group> hg;
  for (auto& g : ctx->groups) {
    const tnmc_config& c = g.cfg;
    if ((st = dalloc(ctx, (void**)&g.d_spins, g.vol * c.n_chains)) != TNMC_OK) { tnmc_destroy(ctx); return st; }
    if ((st = dalloc(ctx, (void**)&g.d_J, sizeof(int32_t) * 3 * g.vol * c.n_inst)) != TNMC_OK) { tnmc_destroy(ctx); return st; }
    if ((st = dalloc(ctx, (void**)&g.d_beta, sizeof(double) * c.n_chains)) != TNMC_OK) { tnmc_destroy(ctx); return st; }
    if ((st = dalloc(ctx, (void**)&g.d_inst, sizeof(int32_t) * c.n_chains)) != TNMC_OK) { tnmc_destroy(ctx); return st; }
    cudaMemsetAsync(g.d_spins, 0, g.vol * c.n_chains, ctx->stream);
    cudaMemcpyAsync(g.d_J, c.couplings, sizeof(int32_t) * 3 * g.vol * c.n_inst,
                    c.couplings_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(g.d_beta, c.betas, sizeof(double) * c.n_chains, cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(g.d_inst, c.instance_of_chain, sizeof(int32_t) * c.n_chains, cudaMemcpyHostToDevice, ctx->stream);
    Group d;
    d.L[0] = c.Lx; d.L[1] = c.Ly; d.L[2] = c.Lz;
    for (int a = 0; a < 3; ++a) d.bc[a] = c.bc[a];
    d.model = c.model; d.d = g.d; d.chi = c.chi; d.fix_mode = c.fix_mode; d.n_chains = c.n_chains;
    d.chain_base = g.chain_base; d.spins = g.d_spins; d.J = g.d_J; d.beta = g.d_beta; d.inst = g.d_inst;
    d.layers = g.cfg.layers;
    // the host copies of betas/instances/couplings are not kept
    g.cfg.betas = nullptr; g.cfg.instance_of_chain = nullptr; g.cfg.couplings = nullptr;
    hg.push_back(d);
  }
  if ((st = dalloc(ctx, (void**)&ctx->d_groups, sizeof(Group) * hg.size())) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  cudaMemcpyAsync(ctx->d_groups, hg.data(), sizeof(Group) * hg.size(), cudaMemcpyHostToDevice, ctx->stream);
  if ((st = dalloc(ctx, (void**)&ctx->d_sweep, sizeof(unsigned long long))) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  if ((st = dalloc(ctx, (void**)&ctx->d_events, sizeof(unsigned long long))) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  if ((st = dalloc(ctx, (void**)&ctx->d_status, sizeof(unsigned int))) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), ctx->stream);
  cudaMemsetAsync(ctx->d_sweep, 0, sizeof(unsigned long long), ctx->stream);
  cudaMemsetAsync(ctx->d_events, 0, sizeof(unsigned long long), ctx->stream);
  // work-list buffer for explicit batches and the logz hook
  int maxit = 1;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) maxit = std::max(maxit, items_for(ctx, a, c));
  for (auto& g : ctx->groups) maxit = std::max(maxit, g.cfg.n_chains * std::max(g.cfg.Lx, std::max(g.cfg.Ly, g.cfg.Lz)));
  ctx->max_items = maxit;
  if ((st = dalloc(ctx, (void**)&ctx->d_items, sizeof(int) * 3 * maxit)) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  if ((st = dalloc(ctx, (void**)&ctx->d_logz, sizeof(double))) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  // per-CTA workspace: as many CTAs as fit on the GPU (2 per SM) within a memory budget
  ctx->lay = ctx->precision == TNMC_PREC_F64 ? make_layout<double>(Mmax, Lmax, dmax, chimax)
                                             : make_layout<float>(Mmax, Lmax, dmax, chimax);
  ctx->ws_stride = ctx->lay.total_bytes;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  // dynamic shared memory: the (d chi) x (d chi) eigenproblem (density-matrix route), or the
  // one-sided Jacobi rows and the LQ panels (LQ route), when they fit
  const size_t rsz = ctx->precision == TNMC_PREC_F64 ? sizeof(double) : sizeof(float);
  const size_t nd = (size_t)dmax * chimax;
  ctx->eig_bytes = nd * (nd + 1) * rsz;
  const size_t zbytes = nd * (nd + 4) * rsz;
  const size_t panbytes = (size_t)32 * dmax * ctx->lay.nmax * rsz;
  ctx->lq_bytes = std::min<size_t>(std::max(zbytes, panbytes), kDynSmemCap);
  ctx->jac_floor = ctx->precision == TNMC_PREC_F64 ? 0 : 1;
  // FP32: CUDA-core FMA by default (measured as fast as 3xTF32 on the tensor cores for these
  // latency-bound per-CTA contractions, and one rounding fewer)
  ctx->gemm_mode = ctx->precision == TNMC_PREC_BF16 ? GEMM_BF16 : GEMM_FFMA;
  int per_sm = apply_smem(ctx);
  per_sm = std::max(1, std::min(per_sm, 2));
  ctx->ctas_per_sm = per_sm;
  ctx->sms = sms;
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  const size_t budget = freeb / 2;
  int ctas = std::min(maxit, sms * per_sm);
  while (ctas > 1 && (size_t)ctas * ctx->ws_stride > budget) --ctas;
  ctx->max_ctas = std::max(1, ctas);
  ctx->alloc_ctas = ctx->max_ctas;
  if ((st = dalloc(ctx, (void**)&ctx->d_ws, ctx->ws_stride * ctx->max_ctas)) != TNMC_OK) { tnmc_destroy(ctx); return st; }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) { tnmc_destroy(ctx); return TNMC_ERR_CUDA; }
  *out = ctx;
  return TNMC_OK;
}

tnmc_status tnmc_set_spins(tnmc_ctx* ctx, int group, const int8_t* spins, int on_device) {
  if (!ctx || !spins || group < 0 || group >= (int)ctx->groups.size()) return fail(ctx, TNMC_ERR_ARG, "set_spins");
  auto& g = ctx->groups[group];
  CU(cudaMemcpyAsync(g.d_spins, spins, g.vol * g.cfg.n_chains,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!on_device) CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

tnmc_status tnmc_get_spins(tnmc_ctx* ctx, int group, int8_t* out, int on_device) {
  if (!ctx || !out || group < 0 || group >= (int)ctx->groups.size()) return fail(ctx, TNMC_ERR_ARG, "get_spins");
  auto& g = ctx->groups[group];
  CU(cudaMemcpyAsync(out, g.d_spins, g.vol * g.cfg.n_chains,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  CU(cudaGetLastError());
  return read_status(ctx);
}

tnmc_status tnmc_slice_update(tnmc_ctx* ctx, int group, int axis, int n_items, const int32_t* chain_ids,
                              const int32_t* slice_ids, uint64_t seed, uint64_t step, int proposal, int write_back,
                              int8_t* new_spins_out, double* logq_new, double* logq_old, uint8_t* accept,
                              int64_t* dE) {
  if (!ctx || group < 0 || group >= (int)ctx->groups.size() || axis < 0 || axis > 2 || n_items < 0 ||
      n_items > ctx->max_items || (n_items && (!chain_ids || !slice_ids)))
    return fail(ctx, TNMC_ERR_ARG, "slice_update: bad argument");
  if (proposal != TNMC_PROPOSAL_TN && proposal != TNMC_PROPOSAL_NET && proposal != TNMC_PROPOSAL_CACHE)
    return fail(ctx, TNMC_ERR_ARG, "slice_update: proposal");
  if (proposal == TNMC_PROPOSAL_CACHE && !ctx->cache_ready)
    return fail(ctx, TNMC_ERR_STATE, "slice_update: no environment cache (call tnmc_cache_build)");
  if (proposal == TNMC_PROPOSAL_NET && !ctx->net_on)
    return fail(ctx, TNMC_ERR_STATE, "slice_update: no proposal network (call tnmc_net_init)");
  if (n_items == 0) return TNMC_OK;
  const auto& g = ctx->groups[group];
  const int L[3] = {g.cfg.Lx, g.cfg.Ly, g.cfg.Lz};
  const int n = L[axis];
  std::vector<std::vector<int>> per(g.cfg.n_chains);
  const bool comp = g.cfg.layers == 2;
  for (int i = 0; i < n_items; ++i) {
    if (chain_ids[i] < 0 || chain_ids[i] >= g.cfg.n_chains || slice_ids[i] < 0 || slice_ids[i] >= n)
      return fail(ctx, TNMC_ERR_ARG, "slice_update: chain or slice out of range");
    if (comp && !g.cfg.bc[axis] && slice_ids[i] + 1 >= n)
      return fail(ctx, TNMC_ERR_ARG, "slice_update: composite layer leaves the lattice on an open axis");
    per[chain_ids[i]].push_back(slice_ids[i]);
  }
  // a slice reaches its neighbours; a composite (k, k+1) reaches k-1 .. k+2, so two composites of one
  // chain must start at least 3 layers apart (cyclically on a periodic axis)
  const int reach = comp ? 2 : 1;
  for (auto& v : per)
    for (size_t a = 0; a < v.size(); ++a)
      for (size_t b = a + 1; b < v.size(); ++b) {
        const int dk = std::abs(v[a] - v[b]);
        if (dk <= reach || (g.cfg.bc[axis] && dk >= n - reach))
          return fail(ctx, TNMC_ERR_ADJACENT, "slice_update: batch holds adjacent or repeated slices of one chain");
      }
  std::vector<int> items(3 * (size_t)n_items);
  for (int i = 0; i < n_items; ++i) {
    items[i] = group;
    items[n_items + i] = chain_ids[i];
    items[2 * n_items + i] = slice_ids[i];
  }
  CU(cudaMemcpyAsync(ctx->d_items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  PhaseParams P{};
  P.item_group = ctx->d_items;
  P.item_chain = ctx->d_items + n_items;
  P.item_slice = ctx->d_items + 2 * n_items;
  P.n_items = n_items;
  P.axis = axis;
  P.step = (uint32_t)step;
  P.seed = seed;
  P.write_back = write_back;
  P.out_spins = new_spins_out;
  P.out_lq_new = logq_new;
  P.out_lq_old = logq_old;
  P.out_acc = accept;
  P.out_dE = dE;
  P.proposal = proposal == TNMC_PROPOSAL_NET ? 1 : 0;
  P.cache_mode = proposal == TNMC_PROPOSAL_CACHE ? CACHE_USE : CACHE_OFF;
  P.record = ctx->record && ctx->net_on;
  launch(ctx, P, n_items);
  CU(cudaGetLastError());
  return TNMC_OK;
}

static void sweep_launches(tnmc_ctx* ctx, cudaStream_t stream, int axis, uint64_t seed, uint32_t* acc) {
  cudaStream_t saved = ctx->stream;
  ctx->stream = stream;
  for (int colour = 0; colour < 3; ++colour) {
    const int total = items_for(ctx, axis, colour);
    if (!total) continue;
    PhaseParams P{};
    P.n_items = -1;
    P.colour = colour;
    P.sweep_ctr = ctx->d_sweep;
    P.seed = seed;
    P.write_back = 1;
    P.acc_counter = acc;
    P.net_every = ctx->net_on ? ctx->net_every : 0;
    P.proposal_ctr = ctx->d_sweep;
    P.record = ctx->record && ctx->net_on;
    P.cache_mode = ctx->cache_on && ctx->cache_ready ? CACHE_SWEEP : CACHE_OFF;
    P.cache_every = ctx->cache_every;
    launch(ctx, P, total);
  }
  bump_sweep<<<1, 1, 0, ctx->stream>>>(ctx->d_sweep);
  ctx->stream = saved;
}

tnmc_status tnmc_sweep(tnmc_ctx* ctx, int n_sweeps, uint64_t seed, int use_graph, uint32_t* accept_out) {
  if (!ctx || n_sweeps < 0) return fail(ctx, TNMC_ERR_ARG, "sweep");
  for (int s = 0; s < n_sweeps; ++s) {
    const int axis = (int)(ctx->h_sweep % 3ull);
    if (use_graph) {
      if (!ctx->graphs[axis] || ctx->graph_seed[axis] != seed || ctx->graph_acc[axis] != accept_out) {
        if (ctx->graphs[axis]) cudaGraphExecDestroy(ctx->graphs[axis]);
        ctx->graphs[axis] = nullptr;
        if (!ctx->cap_stream) CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        // capture on the private stream (the legacy default stream cannot be captured),
        // replay on the context's stream
        cudaGraph_t graph = nullptr;
        CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        sweep_launches(ctx, ctx->cap_stream, axis, seed, accept_out);
        const cudaError_t launch_err = cudaGetLastError();
        const cudaError_t end_err = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (launch_err != cudaSuccess || end_err != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return fail(ctx, TNMC_ERR_CUDA, std::string("sweep capture: ") +
                                              cudaGetErrorString(launch_err != cudaSuccess ? launch_err : end_err));
        }
        const cudaError_t inst_err = cudaGraphInstantiate(&ctx->graphs[axis], graph, 0);
        cudaGraphDestroy(graph);
        if (inst_err != cudaSuccess) {
          ctx->graphs[axis] = nullptr;
          return fail(ctx, TNMC_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(inst_err));
        }
        ctx->graph_seed[axis] = seed;
        ctx->graph_acc[axis] = accept_out;
      }
      CU(cudaGraphLaunch(ctx->graphs[axis], ctx->stream));
    } else {
      sweep_launches(ctx, ctx->stream, axis, seed, accept_out);
    }
    ctx->h_sweep += 1;
  }
  CU(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_get_sweep(tnmc_ctx* ctx, uint64_t* t) {
  if (!ctx || !t) return fail(ctx, TNMC_ERR_ARG, "get_sweep");
  *t = ctx->h_sweep;
  return TNMC_OK;
}

tnmc_status tnmc_set_sweep(tnmc_ctx* ctx, uint64_t t) {
  if (!ctx) return TNMC_ERR_ARG;
  ctx->h_sweep = t;
  unsigned long long v = t;
  CU(cudaMemcpyAsync(ctx->d_sweep, &v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

}  // extern "C"

// observables: one CTA per chain
__global__ void observables_kernel(Group g, const int32_t* partner, double* out) {
  const int c = blockIdx.x;
  __shared__ double red[32];
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  const int8_t* s = g.spins + (size_t)c * vol;
  const int8_t* s2 = g.spins + (size_t)partner[c] * vol;
  const int32_t* J = g.J + (size_t)g.inst[c] * 3 * vol;
  double e = 0.0, m = 0.0, q = 0.0;
  int loc[4] = {0, 0, 0, 0};
  for (size_t i = threadIdx.x; i < vol; i += blockDim.x) {
    const int v = s[i];
    for (int a = 0; a < 3; ++a) {
      const int nb = shift_index(g, (int)i, a, +1);
      e -= (double)J[a * vol + i] * pair_e(g.model, v, s[nb]);
    }
    m += 1 - 2 * v;
    q += (double)((1 - 2 * v) * (1 - 2 * s2[i]));
    if (v < 4) loc[v]++;
  }
  e = block_sum(e, red);
  m = block_sum(m, red);
  q = block_sum(q, red);
  int tot[4];
  for (int v = 0; v < 4; ++v) tot[v] = (int)block_sum((double)loc[v], red);
  if (threadIdx.x == 0) {
    out[c * 3 + 0] = e * kJScale / (double)vol;
    if (g.model == 2) {
      int mx = 0;
      for (int v = 0; v < g.d; ++v) mx = tot[v] > mx ? tot[v] : mx;
      out[c * 3 + 1] = ((double)g.d * mx / (double)vol - 1.0) / (g.d - 1.0);
    } else {
      out[c * 3 + 1] = m / (double)vol;
    }
    out[c * 3 + 2] = q / (double)vol;
  }
}

extern "C" {

tnmc_status tnmc_observables(tnmc_ctx* ctx, int group, const int32_t* partner, double* out) {
  if (!ctx || !out || group < 0 || group >= (int)ctx->groups.size()) return fail(ctx, TNMC_ERR_ARG, "observables");
  auto& g = ctx->groups[group];
  const int n = g.cfg.n_chains;
  std::vector<int32_t> p(n);
  for (int c = 0; c < n; ++c) {
    p[c] = partner ? partner[c] : (c ^ 1);
    if (p[c] < 0 || p[c] >= n) p[c] = c;
  }
  int32_t* dp = ctx->d_items;  // reuse the work-list buffer (n <= max_items)
  CU(cudaMemcpyAsync(dp, p.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
  Group dg;
  CU(cudaMemcpyAsync(&dg, ctx->d_groups + group, sizeof(Group), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  observables_kernel<<<n, kThreads, 0, ctx->stream>>>(dg, dp, out);
  CU(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_slice_logz(tnmc_ctx* ctx, int group, int chain, int axis, int slice, uint64_t seed, uint64_t step,
                            double* logz) {
  if (!ctx || !logz || group < 0 || group >= (int)ctx->groups.size() || axis < 0 || axis > 2)
    return fail(ctx, TNMC_ERR_ARG, "slice_logz");
  const auto& g = ctx->groups[group];
  const int L[3] = {g.cfg.Lx, g.cfg.Ly, g.cfg.Lz};
  if (chain < 0 || chain >= g.cfg.n_chains || slice < 0 || slice >= L[axis]) return fail(ctx, TNMC_ERR_ARG, "slice_logz");
  int items[3] = {group, chain, slice};
  CU(cudaMemcpyAsync(ctx->d_items, items, sizeof(items), cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  PhaseParams P{};
  P.item_group = ctx->d_items;
  P.item_chain = ctx->d_items + 1;
  P.item_slice = ctx->d_items + 2;
  P.n_items = 1;
  P.axis = axis;
  P.step = (uint32_t)step;
  P.seed = seed;
  P.logz_only = 1;
  P.out_logz = ctx->d_logz;
  launch(ctx, P, 1);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(logz, ctx->d_logz, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return read_status(ctx);
}

tnmc_status tnmc_set_proposal_beta_factor(tnmc_ctx* ctx, double factor) {
  if (!ctx || !(factor > 0.0)) return fail(ctx, TNMC_ERR_ARG, "beta factor");
  ctx->env_beta_factor = factor;
  for (auto& gexec : ctx->graphs)
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
  return TNMC_OK;
}

tnmc_status tnmc_metropolis_sweep(tnmc_ctx* ctx, int n_sweeps, uint64_t seed, uint32_t* accept_out) {
  if (!ctx || n_sweeps < 0) return fail(ctx, TNMC_ERR_ARG, "metropolis_sweep");
  std::vector<Group> hg(ctx->groups.size());
  for (size_t gi = 0; gi < ctx->groups.size(); ++gi) {
    const auto& g = ctx->groups[gi];
    const int L[3] = {g.cfg.Lx, g.cfg.Ly, g.cfg.Lz};
    if (g.d != 2) return fail(ctx, TNMC_ERR_ARG, "metropolis_sweep: Ising models only");
    for (int a = 0; a < 3; ++a)
      if (g.cfg.bc[a] && (L[a] & 1))
        return fail(ctx, TNMC_ERR_ARG, "metropolis_sweep: a periodic axis of odd extent is not bipartite");
  }
  CU(cudaMemcpyAsync(hg.data(), ctx->d_groups, sizeof(Group) * hg.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  for (int s = 0; s < n_sweeps; ++s) {
    for (int colour = 0; colour < 2; ++colour)
      for (const auto& g : hg)
        tnmc_launch_metropolis(g, seed, (uint32_t)ctx->h_metro, colour, accept_out, ctx->stream);
    ctx->h_metro += 1;
  }
  CU(cudaGetLastError());
  return TNMC_OK;
}

tnmc_status tnmc_set_proposals_per_env(tnmc_ctx* ctx, int n_prop) {
  if (!ctx || n_prop < 1 || n_prop > 64) return fail(ctx, TNMC_ERR_ARG, "proposals per environment: 1..64");
  ctx->n_prop = n_prop;
  drop_graphs(ctx);
  return TNMC_OK;
}

tnmc_status tnmc_cache_build(tnmc_ctx* ctx, uint64_t seed, uint64_t step) {
  if (!ctx) return TNMC_ERR_ARG;
  for (const auto& g : ctx->groups)
    if (g.cfg.layers == 2) return fail(ctx, TNMC_ERR_ARG, "cache_build: composite-layer groups are not cached");
  if (!ctx->d_cache) {
    // slot: the environment stack as the workspace holds it, the bond dims, then (y0, x0, built)
    const size_t rsz = ctx->precision == TNMC_PREC_F64 ? sizeof(double) : sizeof(float);
    const WsLayout& L = ctx->lay;
    const size_t e_bytes = (size_t)L.Mmax * L.Lmax * L.dmax * L.chimax * L.chimax * rsz;
    const size_t d_bytes = sizeof(int) * (size_t)(L.Mmax + 1) * (L.Lmax + 1);
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    int lmax = 2;
    for (const auto& g : ctx->groups) lmax = std::max(lmax, std::max(g.cfg.Lx, std::max(g.cfg.Ly, g.cfg.Lz)));
    const size_t stride = up(e_bytes) + up(d_bytes) + 256;
    const size_t total = stride * (size_t)ctx->total_chains * 3 * lmax;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    if (total > freeb) return fail(ctx, TNMC_ERR_OOM, "cache_build: the cache does not fit in device memory");
    tnmc_status st = dalloc(ctx, (void**)&ctx->d_cache, total);
    if (st != TNMC_OK) return st;
    ctx->cache_stride = stride;
    ctx->cache_dims_off = up(e_bytes);
    ctx->cache_meta_off = up(e_bytes) + up(d_bytes);
    ctx->cache_lmax = lmax;
    CU(cudaMemsetAsync(ctx->d_cache, 0, total, ctx->stream));
  }
  for (int axis = 0; axis < 3; ++axis) {
    int total = 0;
    for (const auto& g : ctx->groups) {
      const int L[3] = {g.cfg.Lx, g.cfg.Ly, g.cfg.Lz};
      total += L[axis] * g.cfg.n_chains;
    }
    PhaseParams P{};
    P.n_items = -2;
    P.axis = axis;
    P.step = (uint32_t)step;
    P.seed = seed;
    P.cache_mode = CACHE_BUILD;
    launch(ctx, P, total);
    CU(cudaGetLastError());
  }
  ctx->cache_ready = 1;
  drop_graphs(ctx);
  return TNMC_OK;
}

tnmc_status tnmc_set_cache_mix(tnmc_ctx* ctx, int on, int fresh_every) {
  if (!ctx || (on != 0 && on != 1) || fresh_every < 0) return fail(ctx, TNMC_ERR_ARG, "cache_mix");
  if (on && !ctx->cache_ready) return fail(ctx, TNMC_ERR_STATE, "cache_mix: no environment cache (call tnmc_cache_build)");
  ctx->cache_on = on;
  ctx->cache_every = fresh_every;
  drop_graphs(ctx);
  return TNMC_OK;
}

tnmc_status tnmc_sync(tnmc_ctx* ctx) {
  if (!ctx) return TNMC_ERR_ARG;
  CU(cudaStreamSynchronize(ctx->stream));
  CU(cudaGetLastError());
  return read_status(ctx);
}

tnmc_status tnmc_events(tnmc_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return fail(ctx, TNMC_ERR_ARG, "events");
  unsigned long long v = 0;
  CU(cudaMemcpyAsync(&v, ctx->d_events, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  *count = v;
  return TNMC_OK;
}

tnmc_status tnmc_memory(tnmc_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return TNMC_ERR_ARG;
  *bytes = ctx->bytes;
  return TNMC_OK;
}

// Device buffer <-> file section helpers of the checkpoint.
static bool put_dev(FILE* f, const void* dptr, size_t bytes) {
  std::vector<char> buf(bytes);
  if (bytes && cudaMemcpy(buf.data(), dptr, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  return fwrite(buf.data(), 1, bytes, f) == bytes;
}
static bool get_dev(FILE* f, void* dptr, size_t bytes) {
  std::vector<char> buf(bytes);
  if (fread(buf.data(), 1, bytes, f) != bytes) return false;
  return !bytes || cudaMemcpy(dptr, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

// Shape of the learned proposal's state in a checkpoint.
struct NetCkptHeader {
  int32_t d, H, NL, rb_slots, Pmax, net_every, record, adam_t;
  uint64_t n_params, rb_count;
};

tnmc_status tnmc_save(tnmc_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, TNMC_ERR_ARG, "save");
  CU(cudaStreamSynchronize(ctx->stream));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, TNMC_ERR_ARG, "save: cannot open file");
  const char magic[8] = {'T', 'N', 'M', 'C', 'C', 'K', 'P', '2'};
  bool ok = fwrite(magic, 1, 8, f) == 8;
  const uint64_t t = ctx->h_sweep;
  const uint32_t ng = (uint32_t)ctx->groups.size();
  ok = ok && fwrite(&t, sizeof(t), 1, f) == 1 && fwrite(&ng, sizeof(ng), 1, f) == 1;
  for (auto& g : ctx->groups) {
    const uint64_t n = g.vol * g.cfg.n_chains;
    ok = ok && fwrite(&n, sizeof(n), 1, f) == 1 && put_dev(f, g.d_spins, n);
  }
  // learned proposal: weights, Adam moments and step, replay buffer, schedule
  const uint32_t has_net = ctx->net_on ? 1u : 0u;
  ok = ok && fwrite(&has_net, sizeof(has_net), 1, f) == 1;
  if (ok && ctx->net_on) {
    NetCkptHeader h{};
    h.d = ctx->net.d; h.H = ctx->net.H; h.NL = ctx->net.NL; h.rb_slots = ctx->rb_slots; h.Pmax = ctx->Pmax;
    h.net_every = ctx->net_every; h.record = ctx->record; h.adam_t = ctx->adam_t;
    h.n_params = ctx->net.n_params;
    unsigned long long cnt = 0;
    if (cudaMemcpy(&cnt, ctx->d_rb_count, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
    h.rb_count = cnt;
    const size_t np = ctx->net.n_params * sizeof(float);
    ok = ok && fwrite(&h, sizeof(h), 1, f) == 1 && put_dev(f, ctx->d_W, np) && put_dev(f, ctx->d_m1, np) &&
         put_dev(f, ctx->d_m2, np);
    if (ok && ctx->rb_slots > 0) {
      const size_t slots = (size_t)ctx->rb_slots, Pm = (size_t)ctx->Pmax;
      ok = put_dev(f, ctx->d_rb_cond, sizeof(float) * ctx->net.Cc * Pm * slots) &&
           put_dev(f, ctx->d_rb_spins, Pm * slots) && put_dev(f, ctx->d_rb_meta, sizeof(int) * 2 * slots);
    }
  }
  fclose(f);
  return ok ? TNMC_OK : fail(ctx, TNMC_ERR_CUDA, "save: write failed");
}

tnmc_status tnmc_load(tnmc_ctx* ctx, const char* path) {
  if (!ctx || !path) return fail(ctx, TNMC_ERR_ARG, "load");
  CU(cudaStreamSynchronize(ctx->stream));
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, TNMC_ERR_ARG, "load: cannot open file");
  char magic[8];
  uint64_t t = 0;
  uint32_t ng = 0;
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, "TNMCCKP2", 8) || fread(&t, sizeof(t), 1, f) != 1 ||
      fread(&ng, sizeof(ng), 1, f) != 1 || ng != ctx->groups.size()) {
    fclose(f);
    return fail(ctx, TNMC_ERR_ARG, "load: not a checkpoint of this context");
  }
  for (auto& g : ctx->groups) {
    uint64_t n = 0;
    if (fread(&n, sizeof(n), 1, f) != 1 || n != g.vol * g.cfg.n_chains) { fclose(f); return fail(ctx, TNMC_ERR_ARG, "load: size"); }
    if (!get_dev(f, g.d_spins, n)) { fclose(f); return fail(ctx, TNMC_ERR_ARG, "load: truncated"); }
  }
  uint32_t has_net = 0;
  if (fread(&has_net, sizeof(has_net), 1, f) != 1) { fclose(f); return fail(ctx, TNMC_ERR_ARG, "load: truncated"); }
  if (has_net) {
    NetCkptHeader h{};
    if (fread(&h, sizeof(h), 1, f) != 1) { fclose(f); return fail(ctx, TNMC_ERR_ARG, "load: truncated"); }
    if (!ctx->net_on || h.d != ctx->net.d || h.H != ctx->net.H || h.NL != ctx->net.NL ||
        h.n_params != ctx->net.n_params || h.rb_slots != ctx->rb_slots || h.Pmax != ctx->Pmax) {
      fclose(f);
      return fail(ctx, TNMC_ERR_STATE, "load: the checkpoint holds a network; call tnmc_net_init with the same "
                                        "channels, layers and buffer slots first");
    }
    const size_t np = ctx->net.n_params * sizeof(float);
    bool ok = get_dev(f, ctx->d_W, np) && get_dev(f, ctx->d_m1, np) && get_dev(f, ctx->d_m2, np);
    if (ok && ctx->rb_slots > 0) {
      const size_t slots = (size_t)ctx->rb_slots, Pm = (size_t)ctx->Pmax;
      ok = get_dev(f, ctx->d_rb_cond, sizeof(float) * ctx->net.Cc * Pm * slots) &&
           get_dev(f, ctx->d_rb_spins, Pm * slots) && get_dev(f, ctx->d_rb_meta, sizeof(int) * 2 * slots);
    }
    unsigned long long cnt = h.rb_count;
    ok = ok && cudaMemcpy(ctx->d_rb_count, &cnt, sizeof(cnt), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) { fclose(f); return fail(ctx, TNMC_ERR_ARG, "load: truncated network state"); }
    ctx->adam_t = h.adam_t;
    ctx->net_every = h.net_every;
    ctx->record = h.record;
    drop_graphs(ctx);
  }
  fclose(f);
  return tnmc_set_sweep(ctx, t);
}


tnmc_status tnmc_get_tuning(tnmc_ctx* ctx, tnmc_tuning* t) {
  if (!ctx || !t) return TNMC_ERR_ARG;
  t->gemm_mode = ctx->gemm_mode;
  t->eig_smem = ctx->fact_smem ? 1 : 0;
  t->jac_floor = ctx->jac_floor;
  t->ctas_per_sm = ctx->ctas_per_sm;
  t->route = ctx->route;
  t->gemm_tile = ctx->gemm_tile;
  return TNMC_OK;
}

tnmc_status tnmc_set_tuning(tnmc_ctx* ctx, const tnmc_tuning* t) {
  if (!ctx || !t) return TNMC_ERR_ARG;
  // every field is checked before any is applied, so a refused call leaves the context as it was
  const int m = t->gemm_mode;
  if (m >= 0) {
    // F32 keeps FP32-level products (FFMA or a 3xTF32 engine); BF16 takes a BF16 engine; F64 ignores it
    if (m > GEMM_UMMA_BF16) return fail(ctx, TNMC_ERR_ARG, "set_tuning: gemm_mode");
    if (ctx->precision == TNMC_PREC_F32 && m != GEMM_FFMA && m != GEMM_TF32X3 && m != GEMM_UMMA_TF32X3)
      return fail(ctx, TNMC_ERR_ARG, "set_tuning: gemm_mode for F32 must be FFMA or a 3xTF32 engine");
    if (ctx->precision == TNMC_PREC_BF16 && m != GEMM_BF16 && m != GEMM_UMMA_BF16)
      return fail(ctx, TNMC_ERR_ARG, "set_tuning: gemm_mode for BF16 must be a BF16 engine");
  }
  if (t->jac_floor > 2) return fail(ctx, TNMC_ERR_ARG, "set_tuning: jac_floor");
  if (t->route > 1) return fail(ctx, TNMC_ERR_ARG, "set_tuning: route");
  if (t->gemm_tile > 2 || (t->gemm_tile > 0 && ctx->precision == TNMC_PREC_F64))
    return fail(ctx, TNMC_ERR_ARG, "set_tuning: gemm_tile (F32 / BF16: 0, 1 or 2; F64: 0)");
  if (t->ctas_per_sm == 0 || t->ctas_per_sm > 2) return fail(ctx, TNMC_ERR_ARG, "set_tuning: ctas_per_sm");
  if (m >= 0 && ctx->precision != TNMC_PREC_F64) ctx->gemm_mode = m;
  if (t->jac_floor >= 0) ctx->jac_floor = t->jac_floor;
  if (t->route >= 0) ctx->route = t->route;
  if (t->eig_smem >= 0) ctx->smem_on = t->eig_smem ? 1 : 0;
  if (t->gemm_tile >= 0) ctx->gemm_tile = t->gemm_tile;
  if (t->ctas_per_sm >= 0) ctx->req_ctas = t->ctas_per_sm;
  const int occ = apply_smem(ctx);
  // the request, not the last occupancy, decides: an instance of lower occupancy (tcgen05) does not
  // leave the context at one CTA per SM after switching back
  const int want = std::min(ctx->req_ctas, std::max(1, occ));
  // the workspace was sized for the CTA count at creation; never exceed it
  ctx->max_ctas = std::max(1, std::min(ctx->alloc_ctas, ctx->sms * want));
  ctx->ctas_per_sm = want;
  drop_graphs(ctx);
  return TNMC_OK;
}

tnmc_status tnmc_net_init(tnmc_ctx* ctx, int channels, int layers, uint64_t seed, int buffer_slots) {
  if (!ctx || channels < 1 || channels > 64 || layers < 2 || layers > kNetMaxLayers || buffer_slots < 0)
    return fail(ctx, TNMC_ERR_ARG, "net_init");
  if (ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "net_init: network already initialised");
  for (const auto& g : ctx->groups)
    if (g.cfg.layers == 2) return fail(ctx, TNMC_ERR_ARG, "net_init: the network proposes single slices, not composite layers");
  int d = 0;
  for (auto& g : ctx->groups) {
    if (d && g.d != d) return fail(ctx, TNMC_ERR_ARG, "net_init: groups with different local dimension");
    d = g.d;
  }
  ctx->net = make_net_layout(d, channels, layers);
  const NetLayout& N = ctx->net;
  ctx->Pmax = ctx->lay.Lmax * ctx->lay.Lmax;
  const int Pm = ctx->Pmax;
  tnmc_status st;
  const size_t np = N.n_params;
  if ((st = dalloc(ctx, (void**)&ctx->d_W, sizeof(float) * np)) != TNMC_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->d_m1, sizeof(float) * np)) != TNMC_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->d_m2, sizeof(float) * np)) != TNMC_OK) return st;
  ctx->net_ws_stride = (size_t)N.Cc * Pm + 2 * (size_t)N.NL * N.H * Pm + (2 * (size_t)Pm + 3) / 4 + 64;
  if ((st = dalloc(ctx, (void**)&ctx->d_net_ws, sizeof(float) * ctx->net_ws_stride * ctx->max_ctas)) != TNMC_OK) return st;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  ctx->train_ctas = sms;
  ctx->train_ws_stride = 2 * (size_t)N.NL * N.H * Pm + 2 * (size_t)N.H * Pm + (size_t)N.Cc * Pm + Pm / 4 + 64;
  if ((st = dalloc(ctx, (void**)&ctx->d_train_ws, sizeof(float) * ctx->train_ws_stride * ctx->train_ctas)) != TNMC_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->d_gbuf, sizeof(float) * np * ctx->train_ctas)) != TNMC_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->d_loss, sizeof(double) * ctx->train_ctas)) != TNMC_OK) return st;
  ctx->max_batch = std::max(ctx->max_items, 4096);
  if ((st = dalloc(ctx, (void**)&ctx->d_slots, sizeof(int) * ctx->max_batch)) != TNMC_OK) return st;
  ctx->rb_slots = buffer_slots;
  if (buffer_slots > 0) {
    if ((st = dalloc(ctx, (void**)&ctx->d_rb_cond, sizeof(float) * N.Cc * (size_t)Pm * buffer_slots)) != TNMC_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->d_rb_spins, (size_t)Pm * buffer_slots)) != TNMC_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->d_rb_meta, sizeof(int) * 2 * buffer_slots)) != TNMC_OK) return st;
    CU(cudaMemsetAsync(ctx->d_rb_meta, 0, sizeof(int) * 2 * buffer_slots, ctx->stream));
  }
  if ((st = dalloc(ctx, (void**)&ctx->d_rb_count, sizeof(unsigned long long))) != TNMC_OK) return st;
  CU(cudaMemsetAsync(ctx->d_rb_count, 0, sizeof(unsigned long long), ctx->stream));
  CU(cudaMemsetAsync(ctx->d_m1, 0, sizeof(float) * np, ctx->stream));
  CU(cudaMemsetAsync(ctx->d_m2, 0, sizeof(float) * np, ctx->stream));
  net_init_kernel<<<256, 256, 0, ctx->stream>>>(N, ctx->d_W, seed);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->adam_t = 0;
  ctx->net_on = true;
  drop_graphs(ctx);
  return TNMC_OK;
}

tnmc_status tnmc_net_param_count(tnmc_ctx* ctx, size_t* n) {
  if (!ctx || !n) return TNMC_ERR_ARG;
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  *n = ctx->net.n_params;
  return TNMC_OK;
}

tnmc_status tnmc_net_set_params(tnmc_ctx* ctx, const float* w, int on_device) {
  if (!ctx || !w) return TNMC_ERR_ARG;
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  CU(cudaMemcpyAsync(ctx->d_W, w, sizeof(float) * ctx->net.n_params,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

tnmc_status tnmc_net_get_params(tnmc_ctx* ctx, float* w, int on_device) {
  if (!ctx || !w) return TNMC_ERR_ARG;
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  CU(cudaMemcpyAsync(w, ctx->d_W, sizeof(float) * ctx->net.n_params,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

tnmc_status tnmc_set_proposal_mix(tnmc_ctx* ctx, int net_every, int record) {
  if (!ctx || net_every < 0) return TNMC_ERR_ARG;
  if ((net_every || record) && !ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  if (record && ctx->rb_slots == 0) return fail(ctx, TNMC_ERR_STATE, "no replay buffer");
  ctx->net_every = net_every;
  ctx->record = record ? 1 : 0;
  drop_graphs(ctx);
  return TNMC_OK;
}

tnmc_status tnmc_net_buffer_count(tnmc_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return TNMC_ERR_ARG;
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  unsigned long long v = 0;
  CU(cudaMemcpyAsync(&v, ctx->d_rb_count, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  *count = v;
  return TNMC_OK;
}

tnmc_status tnmc_net_train(tnmc_ctx* ctx, int n_steps, int batch, float lr, uint64_t seed, double* losses) {
  if (!ctx || n_steps < 0 || batch < 1 || !(lr >= 0.0f)) return fail(ctx, TNMC_ERR_ARG, "net_train");
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  if (batch > ctx->max_batch) return fail(ctx, TNMC_ERR_ARG, "net_train: batch too large");
  // the filled slots (a slot stays empty until an accepted slice is recorded in it)
  std::vector<int> meta(2 * (size_t)ctx->rb_slots);
  CU(cudaMemcpyAsync(meta.data(), ctx->d_rb_meta, sizeof(int) * meta.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  std::vector<int> filled;
  for (int i = 0; i < ctx->rb_slots; ++i)
    if (meta[2 * (size_t)i] > 0 && meta[2 * (size_t)i + 1] > 0) filled.push_back(i);
  if (filled.empty()) return fail(ctx, TNMC_ERR_STATE, "net_train: replay buffer empty");
  const uint64_t avail = filled.size();
  std::vector<int> slots(batch);
  std::vector<double> lp(ctx->train_ctas);
  for (int t = 0; t < n_steps; ++t) {
    for (int b = 0; b < batch; ++b) {
      const double u = philox_uniform(seed, 8u, (uint32_t)b, (uint32_t)ctx->adam_t, 0, (uint32_t)t, 0);
      slots[b] = filled[(size_t)std::min<uint64_t>((uint64_t)(u * (double)avail), avail - 1)];
    }
    CU(cudaMemcpyAsync(ctx->d_slots, slots.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, ctx->stream));
    NetTrainParams T{};
    T.net = ctx->net;
    T.W = ctx->d_W;
    T.gbuf = ctx->d_gbuf;
    T.loss_part = ctx->d_loss;
    T.ws = ctx->d_train_ws;
    T.ws_stride = ctx->train_ws_stride;
    T.Pmax = ctx->Pmax;
    T.rb_cond = ctx->d_rb_cond;
    T.rb_spins = ctx->d_rb_spins;
    T.rb_meta = ctx->d_rb_meta;
    T.slots = ctx->d_slots;
    T.batch = batch;
    T.want_grad = 1;
    const int grid = std::min(batch, ctx->train_ctas);
    net_train_kernel<<<grid, kThreads, 0, ctx->stream>>>(T);
    ctx->adam_t += 1;
    net_adam_kernel<<<256, 256, 0, ctx->stream>>>(ctx->net.n_params, ctx->d_W, ctx->d_m1, ctx->d_m2, ctx->d_gbuf,
                                                  grid, lr, 0.9f, 0.999f, 1e-8f, ctx->adam_t, nullptr);
    CU(cudaGetLastError());
    if (losses) {
      CU(cudaMemcpyAsync(lp.data(), ctx->d_loss, sizeof(double) * grid, cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
      double tot = 0.0;
      for (int i = 0; i < grid; ++i) tot += lp[i];
      losses[t] = tot / batch;
    }
  }
  CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

tnmc_status tnmc_net_adam_step(tnmc_ctx* ctx, const float* grad, int on_device, float lr) {
  if (!ctx || !grad || !(lr >= 0.0f)) return fail(ctx, TNMC_ERR_ARG, "net_adam_step");
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  CU(cudaMemcpyAsync(ctx->d_gbuf, grad, sizeof(float) * ctx->net.n_params,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  ctx->adam_t += 1;
  net_adam_kernel<<<256, 256, 0, ctx->stream>>>(ctx->net.n_params, ctx->d_W, ctx->d_m1, ctx->d_m2, ctx->d_gbuf, 1, lr,
                                                0.9f, 0.999f, 1e-8f, ctx->adam_t, nullptr);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

tnmc_status tnmc_net_eval(tnmc_ctx* ctx, int group, int axis, int n_items, const int32_t* chain_ids,
                          const int32_t* slice_ids, uint64_t seed, uint64_t step, float* logits_out, double* logq_out,
                          float* grad_out) {
  if (!ctx || group < 0 || group >= (int)ctx->groups.size() || axis < 0 || axis > 2 || n_items < 1 ||
      n_items > ctx->max_batch || !chain_ids || !slice_ids)
    return fail(ctx, TNMC_ERR_ARG, "net_eval");
  if (!ctx->net_on) return fail(ctx, TNMC_ERR_STATE, "no network");
  const auto& g = ctx->groups[group];
  const int L[3] = {g.cfg.Lx, g.cfg.Ly, g.cfg.Lz};
  std::vector<int> items(3 * (size_t)n_items);
  for (int i = 0; i < n_items; ++i) {
    if (chain_ids[i] < 0 || chain_ids[i] >= g.cfg.n_chains || slice_ids[i] < 0 || slice_ids[i] >= L[axis])
      return fail(ctx, TNMC_ERR_ARG, "net_eval: chain or slice out of range");
    items[i] = group;
    items[n_items + i] = chain_ids[i];
    items[2 * n_items + i] = slice_ids[i];
  }
  if (n_items > ctx->max_items) return fail(ctx, TNMC_ERR_ARG, "net_eval: too many items");
  CU(cudaMemcpyAsync(ctx->d_items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice, ctx->stream));
  NetTrainParams T{};
  T.net = ctx->net;
  T.W = ctx->d_W;
  T.gbuf = grad_out ? ctx->d_gbuf : nullptr;
  T.loss_part = nullptr;
  T.ws = ctx->d_train_ws;
  T.ws_stride = ctx->train_ws_stride;
  T.Pmax = ctx->Pmax;
  T.batch = n_items;
  T.groups = ctx->d_groups;
  T.item_group = ctx->d_items;
  T.item_chain = ctx->d_items + n_items;
  T.item_slice = ctx->d_items + 2 * n_items;
  T.axis = axis;
  T.step = (uint32_t)step;
  T.seed = seed;
  T.logits_out = logits_out;
  T.logq_out = logq_out;
  T.want_grad = grad_out ? 1 : 0;
  const int grid = std::min(n_items, ctx->train_ctas);
  net_train_kernel<<<grid, kThreads, 0, ctx->stream>>>(T);
  if (grad_out)
    net_adam_kernel<<<256, 256, 0, ctx->stream>>>(ctx->net.n_params, ctx->d_W, ctx->d_m1, ctx->d_m2, ctx->d_gbuf,
                                                  grid, 0.0f, 0.9f, 0.999f, 1e-8f, 1, grad_out);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(ctx->stream));
  return TNMC_OK;
}

const char* tnmc_last_error(const tnmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void tnmc_destroy(tnmc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& gexec : ctx->graphs)
    if (gexec) cudaGraphExecDestroy(gexec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (auto& g : ctx->groups) {
    cudaFree(g.d_spins); cudaFree(g.d_J); cudaFree(g.d_beta); cudaFree(g.d_inst);
  }
  cudaFree(ctx->d_groups); cudaFree(ctx->d_sweep); cudaFree(ctx->d_events); cudaFree(ctx->d_status);
  cudaFree(ctx->d_items);
  cudaFree(ctx->d_logz); cudaFree(ctx->d_ws);
  cudaFree(ctx->d_W); cudaFree(ctx->d_m1); cudaFree(ctx->d_m2); cudaFree(ctx->d_net_ws); cudaFree(ctx->d_train_ws);
  cudaFree(ctx->d_gbuf); cudaFree(ctx->d_loss); cudaFree(ctx->d_slots); cudaFree(ctx->d_rb_cond);
  cudaFree(ctx->d_rb_spins); cudaFree(ctx->d_rb_meta); cudaFree(ctx->d_rb_count);
  cudaFree(ctx->d_cache);
  delete ctx;
}

}  // extern "C"

#ifdef TNMC_PROFILE
// Profiling builds only: per-phase cycle sums accumulated by thread 0 of every CTA; read and reset.
// 0 right sweep (8 its GEMMs, 4 the assembly of N_x), 1 left sweep (9 G' and Y, 10 the P and Z
// GEMMs, 7 the assembly of rho, 2 eigensolves, 11 ranking and the G_new GEMMs), 3 sampling,
// 5 Jacobi sweeps and 6 eigensolves (counts).
extern "C" int tnmc_prof_read(unsigned long long* out) {
  cudaDeviceSynchronize();
  unsigned long long a[16], b[16];
  tnmc::slice_prof_read<float>(a);
  tnmc::slice_prof_read<double>(b);
  for (int i = 0; i < 16; ++i) out[i] = a[i] + b[i];
  return 0;
}
#endif
