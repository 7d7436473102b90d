// Barrier evaluation without any device allocation.
//
// sim_eval_barrier allocates its scratch (the preconditioner diagonal and
// Dirichlet buffers the barrier kernel also fills, the pair count) with
// cudaMalloc on every call.  Some callers cannot allocate device memory once
// they are running: a control loop on a fixed memory budget, or a process in
// which another allocator owns the device memory.  sim_eval_barrier_noalloc
// computes the same result with its scratch in the file-scope device array
// below, whose size is fixed when the library is loaded.
#include <mutex>
#include <string>
#include "../../include/ipcsim.h"
#include "common.cuh"
#include "kernels.h"

namespace {

// 2^20 doubles (8 MiB) on every GPU that loads this library, held until the process exits.
constexpr size_t kNoallocScratchDoubles = size_t(1) << 20;
__device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

// Defined in sim.cu: the pieces of the simulator this entry point reads.
ipc_status sim_internal_scene(ipcsim* sim, const ipc::DevScene** S, void** stream, double* sh, double* kappa,
                              std::string** err);

extern "C" ipc_status sim_eval_barrier_noalloc(ipcsim* sim, const double* x_dev, int n, const int* rec_dev,
                                               int project, double* E_dev, double* grad_dev, double* H_dev) {
  if (!sim || !x_dev || n < 0 || (n && !rec_dev) || !E_dev || !grad_dev || (n && !H_dev)) return IPC_ERR_ARG;
  const ipc::DevScene* S = nullptr;
  void* stream = nullptr;
  double sh = 0, kappa = 0;
  std::string* err = nullptr;
  ipc_status s = sim_internal_scene(sim, &S, &stream, &sh, &kappa, &err);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nk = S->nk > 0 ? S->nk : 1;
  // layout in 8-byte slots: [count | E (3) | Dc (n_nodes, 9, 3) | gdir (n_nodes, 3, 3) | grad (n_nodes, 3, 3) |
  // pD (nk, 3)]; the sums are order-independent accumulators of three words per value
  const size_t need = 4 + (27 + 9 + 9) * (size_t)S->n_nodes + 3 * nk;
  if (need > kNoallocScratchDoubles) {
    *err = "sim_eval_barrier_noalloc: this scene needs " + std::to_string(need) +
           " scratch slots, more than the " + std::to_string(kNoallocScratchDoubles) +
           " of the static buffer (at most about " + std::to_string((kNoallocScratchDoubles - 8) / 48) +
           " nodes); use sim_eval_barrier";
    return IPC_ERR_ARG;
  }
  double* base = nullptr;
  cudaError_t ce = scratch_address(&base);
  if (ce != cudaSuccess) {
    *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce);
    return IPC_ERR_CUDA;
  }
  int* n_dev = reinterpret_cast<int*>(base);
  ipc::acc_t* Eacc = reinterpret_cast<ipc::acc_t*>(base + 1);
  ipc::acc_t* Dc = Eacc + 3;
  ipc::acc_t* gdir = Dc + 27 * (size_t)S->n_nodes;
  ipc::acc_t* gacc = gdir + 9 * (size_t)S->n_nodes;
  double* pD = reinterpret_cast<double*>(gacc + 9 * (size_t)S->n_nodes);
  // the array keeps the previous call's contents: clear what is accumulated into
  int n_host = n;
  ce = cudaMemcpyAsync(n_dev, &n_host, sizeof(int), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(base + 1, 0, sizeof(double) * (need - 1), st);
  if (ce != cudaSuccess) {
    *err = std::string("sim_eval_barrier_noalloc: ") + cudaGetErrorString(ce);
    return IPC_ERR_CUDA;
  }
  // mode 2 (gradient and Hessian) launches one warp per pair and sizes that grid itself
  ipc::launch_barrier(st, 1, *S, x_dev, rec_dev, n_dev, n, sh, kappa, 1.0, 2, project, gacc, H_dev, Dc, pD, gdir, Eacc,
                      nullptr);
  ipc::launch_acc_finalize(st, 3 * (size_t)S->n_nodes, gacc, nullptr, grad_dev);
  ipc::launch_acc_finalize(st, 1, Eacc, nullptr, E_dev);
  ce = cudaStreamSynchronize(st);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    *err = std::string("sim_eval_barrier_noalloc: ") + cudaGetErrorString(ce);
    return IPC_ERR_CUDA;
  }
  return IPC_OK;
}
