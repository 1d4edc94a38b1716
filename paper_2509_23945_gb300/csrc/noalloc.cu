// tnmc_slice_logz_noalloc: the slice log Z computation of tnmc_slice_logz for
// callers that cannot allocate device memory.
//
// Some hosts own every byte of device memory and forbid raw allocations from
// plugins: frameworks that run all device work through their own arena or
// memory pool, or real-time services that allocate once at start-up and must
// not call cudaMalloc afterwards. Such callers cannot create a tnmc context
// (which allocates its workspace). This entry point needs no context: the
// caller passes the spins, couplings and output on the device, and the
// kernel's scratch lives in a fixed file-scope device array of this library.
//
// Limits: lattice extents <= kNaMaxL, chi <= kNaMaxChi, Ising models only
// (d = 2), FP64 arithmetic. The scratch array (kScratchBytes) is reserved on
// every GPU that loads the library, for the life of the process.
#include <cmath>
#include <mutex>

#include "../../include/tnmc.h"
#include "common.cuh"
#include "slice_launch.cuh"

using namespace tnmc;

namespace {

constexpr int kNaMaxL = 16;
constexpr int kNaMaxChi = 16;
constexpr int kNaMaxD = 2;
constexpr size_t kScratchBytes = size_t(2) << 20;   // 2 MiB, checked against the layout below
constexpr int kMaxDevices = 64;

struct NaHeader {
  Group group;
  double beta;
  int32_t inst;
  int items[3];
};

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
void* g_header_ptr[kMaxDevices] = {nullptr};

}  // namespace

// The scratch: the per-CTA workspace of one slice (environments, right
// factors, GEMM operands) plus a small header with the lattice descriptor.
// Both are shared by every call on a device.
static __device__ __align__(256) unsigned char tnmc_noalloc_scratch[kScratchBytes];
static __device__ __align__(256) NaHeader tnmc_noalloc_header;

// Writes the call's header into the device array. The header travels as a kernel
// argument, so the copy is ordered on the caller's stream and refers to no host memory.
static __global__ void noalloc_write_header(NaHeader hd) { tnmc_noalloc_header = hd; }

extern "C" tnmc_status tnmc_slice_logz_noalloc(const int8_t* spins, const int32_t* couplings, int Lx, int Ly,
                                               int Lz, const int* bc, int model, double beta, int chi, int axis,
                                               int slice, uint64_t seed, uint64_t step, int fix_mode,
                                               double* logz_out, void* cuda_stream) {
  if (!spins || !couplings || !bc || !logz_out) return TNMC_ERR_ARG;
  const int L[3] = {Lx, Ly, Lz};
  for (int a = 0; a < 3; ++a)
    if (L[a] < 2 || L[a] > kNaMaxL || (bc[a] != 0 && bc[a] != 1)) return TNMC_ERR_ARG;
  if (model != TNMC_MODEL_EA_PM && model != TNMC_MODEL_EA_GAUSS) return TNMC_ERR_ARG;  // d = 2 only
  if (chi < 1 || chi > kNaMaxChi || axis < 0 || axis > 2 || slice < 0 || slice >= L[axis]) return TNMC_ERR_ARG;
  if (fix_mode != TNMC_FIX_R1 && fix_mode != TNMC_FIX_R2) return TNMC_ERR_ARG;
  if (!std::isfinite(beta) || beta < 0.0) return TNMC_ERR_ARG;
  const WsLayout lay = make_layout<double>(kNaMaxL, kNaMaxL, kNaMaxD, kNaMaxChi);
  if (lay.total_bytes > kScratchBytes) return TNMC_ERR_STATE;  // build-time sizing error
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TNMC_ERR_CUDA;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  {
    // first call on this device: resolve the device addresses of the scratch
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* s = nullptr;
      void* h = nullptr;
      if (cudaGetSymbolAddress(&s, tnmc_noalloc_scratch) != cudaSuccess) return TNMC_ERR_CUDA;
      if (cudaGetSymbolAddress(&h, tnmc_noalloc_header) != cudaSuccess) return TNMC_ERR_CUDA;
      g_scratch_ptr[dev] = s;
      g_header_ptr[dev] = h;
    }
  }
  NaHeader hd{};
  NaHeader* dh = reinterpret_cast<NaHeader*>(g_header_ptr[dev]);
  hd.group.L[0] = Lx; hd.group.L[1] = Ly; hd.group.L[2] = Lz;
  for (int a = 0; a < 3; ++a) hd.group.bc[a] = bc[a];
  hd.group.model = model;
  hd.group.d = 2;
  hd.group.chi = chi;
  hd.group.fix_mode = fix_mode;
  hd.group.n_chains = 1;
  hd.group.chain_base = 0;
  hd.group.spins = const_cast<int8_t*>(spins);
  hd.group.J = couplings;
  hd.group.beta = &dh->beta;
  hd.group.inst = &dh->inst;
  hd.beta = beta;
  hd.inst = 0;
  hd.items[0] = 0;
  hd.items[1] = 0;
  hd.items[2] = slice;
  // the header travels with a launch on the caller's stream (no allocation, no host pointer kept);
  // an error left by an unrelated earlier call must not be taken for this launch's
  (void)cudaGetLastError();
  noalloc_write_header<<<1, 1, 0, stream>>>(hd);
  if (cudaGetLastError() != cudaSuccess) return TNMC_ERR_CUDA;
  PhaseParams P{};
  P.groups = &dh->group;
  P.n_groups = 1;
  P.item_group = &dh->items[0];
  P.item_chain = &dh->items[1];
  P.item_slice = &dh->items[2];
  P.n_items = 1;
  P.axis = axis;
  P.step = (uint32_t)step;
  P.seed = seed;
  P.env_beta_factor = 1.0;
  P.logz_only = 1;
  P.out_logz = logz_out;
  P.eig_smem = 0;      // no dynamic shared memory: the factorisations stage in the scratch
  P.route = ROUTE_LQ;
  P.dyn_bytes = 0;
  P.jac_floor = 0;
  P.ws = reinterpret_cast<char*>(g_scratch_ptr[dev]);
  P.ws_stride = lay.total_bytes;
  P.lay = lay;
  slice_launch<double>(P, 1, 1, 0, stream);
  if (cudaGetLastError() != cudaSuccess) return TNMC_ERR_CUDA;
  return TNMC_OK;
}
