// Allocation-free contact check.
//
// casim_contacts_noalloc runs the same spatial-hash broad phase and exact
// narrow phase as a casim_step iteration, but keeps every intermediate buffer
// (packed positions, hash counts and offsets, the hash entries, control words)
// in one file-scope device array instead of memory from cudaMalloc.  It exists
// for callers that cannot allocate device memory while they run: real-time
// controllers that must not allocate inside a control loop, and host programs
// whose own allocator owns the GPU's memory pool and forbids outside cudaMalloc
// calls.  The caller still provides the inputs and the outputs.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "casim.h"
#include "common.cuh"
#include "kernels.h"

namespace casim {
namespace {

constexpr int NA_MAX_VERTS = 32768;
constexpr int NA_MAX_TETS = 65536;
constexpr int NA_MAX_QUERY = 16384;
constexpr unsigned NA_HASH = 131072;  // power of two >= 2 * NA_MAX_TETS
constexpr int NA_CAP_ITEMS = 16 * NA_MAX_TETS + 4096;

// Byte offsets of the pieces inside the scratch array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_CTRL = 0;
constexpr size_t OFF_HIST = align256(OFF_CTRL + sizeof(Ctrl));
constexpr size_t OFF_X = align256(OFF_HIST + sizeof(IterRec));
constexpr size_t OFF_COUNT = align256(OFF_X + sizeof(R4<float>) * NA_MAX_VERTS);
constexpr size_t OFF_START = align256(OFF_COUNT + sizeof(int) * (NA_HASH + 2));
constexpr size_t OFF_CURSOR = align256(OFF_START + sizeof(int) * (NA_HASH + 2));
constexpr size_t OFF_ITEMS = align256(OFF_CURSOR + sizeof(int) * (NA_HASH + 1));
constexpr size_t OFF_TILES = align256(OFF_ITEMS + sizeof(int) * NA_CAP_ITEMS);
constexpr size_t OFF_TOTAL = align256(OFF_TILES + sizeof(int) * 1024);
constexpr size_t OFF_OBS = align256(OFF_TOTAL + sizeof(int));
constexpr size_t SCRATCH_BYTES = align256(OFF_OBS + sizeof(int) * NA_MAX_QUERY);

// The scratch: about 6.2 MiB, held by every GPU that loads the library until
// the process exits.  Every call uses all of it, so calls whose GPU work
// overlaps (on different streams or host threads) race with each other.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch per device, looked up once per device with that
// device current.  In host code the name g_scratch is only a host-side stand-in
// and must never be passed to a kernel.  The cached address belongs to the
// device's primary context: it does not survive cudaDeviceReset (the module is
// loaded again in the new context).
std::mutex g_mu;
void* g_addr[64] = {nullptr};

// Control word and statistics record at the start of a call: zero, except the
// bounding-box words, which start at the empty box (as a casim_step iteration
// starts them) so that their atomic min / max reduce to the items' box.
__global__ void k_init_ctrl(Ctrl* ctrl, IterRec* hist) {
  if (threadIdx.x != 0) return;
  Ctrl c{};
  for (int j = 0; j < 3; ++j) {
    c.box_lo[j] = 0x7FFFFFFFFFFFFFFFLL;
    c.box_hi[j] = (long long)0x8000000000000000ULL;
  }
  *ctrl = c;
  *hist = IterRec{};
}

__global__ void k_pack_and_check(const float* xyz, int n_verts, const int* tets, int n_tets, const int* query,
                                 int n_query, R4<float>* X, Ctrl* ctrl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_verts) X[i] = R4<float>{xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.0f};
  if (i < 4 * n_tets) {
    const int v = tets[i];
    if (v < 0 || v >= n_verts) atomicOr(&ctrl->status, ST_BAD_INPUT);
  }
  if (i < n_query) {
    const int v = query[i];
    if (v < 0 || v >= n_verts) atomicOr(&ctrl->status, ST_BAD_INPUT);
  }
}

// Records the reason of a rejection for casim_last_error(NULL) on this thread.
int fail(int code, const std::string& msg) {
  set_handle_free_error(msg.c_str());
  return code;
}

}  // namespace
}  // namespace casim

using namespace casim;

extern "C" int casim_contacts_noalloc(int32_t n_verts, const float* dev_xyz, int32_t n_tets, const int32_t* dev_tets,
                                      int32_t n_query, const int32_t* dev_query, double cell_size,
                                      int32_t max_pairs, int32_t* dev_pair_count, int32_t* dev_pair_tet,
                                      void* cuda_stream) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (n_verts < 1 || n_verts > NA_MAX_VERTS)
    return fail(CASIM_E_INVALID, "n_verts must be in 1.." + std::to_string(NA_MAX_VERTS));
  if (n_tets < 1 || n_tets > NA_MAX_TETS)
    return fail(CASIM_E_INVALID, "n_tets must be in 1.." + std::to_string(NA_MAX_TETS));
  if (n_query < 0 || n_query > NA_MAX_QUERY)
    return fail(CASIM_E_INVALID, "n_query must be in 0.." + std::to_string(NA_MAX_QUERY));
  if (max_pairs < 1 || max_pairs > 16) return fail(CASIM_E_INVALID, "max_pairs must be in 1..16");
  if (!(cell_size > 0.0) || !(cell_size < 1e300)) return fail(CASIM_E_INVALID, "cell_size must be positive");
  if (!dev_xyz || !dev_tets || (n_query > 0 && (!dev_query || !dev_pair_count || !dev_pair_tet)))
    return fail(CASIM_E_INVALID, "null device pointer");
  if (reinterpret_cast<uintptr_t>(dev_tets) % 16 != 0)
    return fail(CASIM_E_INVALID, "dev_tets must be 16-byte aligned");
  if (n_query == 0) return CASIM_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fail(CASIM_E_CUDA, "cudaGetDevice failed");
  if (!g_addr[dev]) {
    // first call on this device: look up the scratch's device address (must
    // happen outside stream capture)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return fail(CASIM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_addr[dev]);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + OFF_CTRL);
  IterRec* hist = reinterpret_cast<IterRec*>(base + OFF_HIST);
  R4<float>* X = reinterpret_cast<R4<float>*>(base + OFF_X);
  // the control word and the statistics record start from their initial values
  k_init_ctrl<<<1, 32, 0, st>>>(ctrl, hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CASIM_E_CUDA, std::string("control init: ") + cudaGetErrorString(e));
  int n_check = n_verts > 4 * n_tets ? n_verts : 4 * n_tets;
  if (n_query > n_check) n_check = n_query;
  k_pack_and_check<<<(n_check + 255) / 256, 256, 0, st>>>(dev_xyz, n_verts, dev_tets, n_tets, dev_query, n_query, X,
                                                          ctrl);
  int status = 0;
  e = cudaMemcpyAsync(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CASIM_E_CUDA, std::string("input check: ") + cudaGetErrorString(e));
  if (status & ST_BAD_INPUT) return fail(CASIM_E_INVALID, "a tet or query vertex id is out of range");

  Dev<float> d{};
  d.n_v = n_verts;
  d.n_t = n_tets;
  d.n_f = 0;
  d.n_q = n_query;
  d.X = X;
  d.tet = reinterpret_cast<const int4*>(dev_tets);
  d.q_verts = dev_query;
  d.H_t = NA_HASH;
  d.H_f = 1;
  d.cell_count = reinterpret_cast<int*>(base + OFF_COUNT);
  d.cell_start = reinterpret_cast<int*>(base + OFF_START);
  d.cell_cursor = reinterpret_cast<int*>(base + OFF_CURSOR);
  d.items = reinterpret_cast<int*>(base + OFF_ITEMS);
  d.cap_items = NA_CAP_ITEMS;
  d.pair_count = dev_pair_count;
  d.pair_tet = dev_pair_tet;
  d.obs_sphere = reinterpret_cast<int*>(base + OFF_OBS);
  d.max_pairs = max_pairs;
  d.collision = 1;
  d.n_spheres = 0;
  d.narrow_threads = 256;  // the regular narrow-phase launch shape; d.sp stays empty: no spring update
  d.cell = cell_size;
  d.inv_cell = 1.0 / cell_size;
  d.ctrl = ctrl;
  d.hist = hist;
  d.hist_cap = 1;
  CollisionScratch cs{reinterpret_cast<int*>(base + OFF_TILES), reinterpret_cast<int*>(base + OFF_TOTAL)};
  launch_collision<float>(d, cs, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CASIM_E_CUDA, std::string("contact check: ") + cudaGetErrorString(e));
  if (status & ST_NONFINITE) return fail(CASIM_E_NONFINITE, "non-finite position");
  if (status & ST_PAIRS_TRUNC)
    return fail(CASIM_E_OVERFLOW, "a query vertex lies in more than max_pairs tets (the smallest ids are kept)");
  if (status & ST_OVERFLOW)
    return fail(CASIM_E_OVERFLOW, "more hash entries than the scratch holds (cell_size too small for the tets)");
  return CASIM_OK;
}
