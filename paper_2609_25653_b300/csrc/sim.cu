// Host orchestration and the C ABI of ipcsim (declared in include/ipcsim.h).
//
// One step (Eq. 3, §III-C.2): predictor and kinematic targets; friction lag
// at x_t; then Newton iterations, each assembling gradient and PSD-projected
// Hessian (inertia, Neo-Hookean, stitch, ABD, barrier, friction), solving
// H_FF p_F = -(g_F + H_FD p_D) by block-Jacobi PCG, bounding the step by
// additive CCD and backtracking on the incremental potential.  Kinematic
// vertices are Dirichlet: p_D = x^_D - x_D moves them with the same step
// fraction; while p_D != 0 the CCD-feasible step is taken without the
// energy test, and a full step snaps them onto their targets.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <thread>
#include <vector>
#include "../../include/ipcsim.h"
#include "common.cuh"
#include "kernels.h"

using namespace ipc;

namespace ipc {
unsigned long long g_kernel_launches = 0;
}

namespace {
thread_local std::string g_create_error;  // reason of the last failed sim_create on this thread
}  // namespace

struct ipcsim {
  ipc_params P{};
  cudaStream_t st = nullptr;
  std::string err;
  DevAlloc mem;                                   // the caller's allocator, or cudaMalloc
  std::vector<std::pair<void*, size_t>> allocs;   // every device block this simulator holds

  // host copies
  int nf = 0, nt = 0, nab = 0, nkb = 0, nv = 0, na_v = 0, nk = 0, n_nodes = 0, nbody = 0;
  std::vector<int> h_sv, h_tris, h_edges;
  double kappa = 0, k_c = 0, L = 0, sh = 0;
  int n_scenes = 1;
  double grav[3] = {0, 0, 0};
  int nnzb = 0;
  std::vector<double> h_Tcur;  // (nkb, 12) current kinematic transforms
  std::vector<double> h_nu, h_logE;  // per-tet material
  double* d_mu = nullptr;
  double* d_lam = nullptr;

  DevScene S{};
  // state
  double *z = nullptr, *zd = nullptr, *xk = nullptr;
  // step work
  double *z_t = nullptr, *z_tilde = nullptr, *xk_t = nullptr, *xk_hat = nullptr, *stitch_hat = nullptr;
  double *xv = nullptr, *xv_t = nullptr, *xv_trial = nullptr, *z_trial = nullptr, *xk_trial = nullptr;
  double *g = nullptr, *gdir = nullptr, *rhs = nullptr, *p = nullptr, *pD = nullptr, *pv = nullptr;
  double *Hconst = nullptr, *Hval = nullptr, *Dc = nullptr, *Dinv = nullptr;
  double *el_tU = nullptr, *el_tG = nullptr;  // per-tet elastic Hessian (upper triangle) and gradient
  int pcg_max_replace = 10;                    // true-residual restarts of a PCG solve
  int nfb = 0;                                 // FEM BSR blocks (rows of the FEM nodes come first)
  // order-independent accumulators of one assembly: gradient, BSR values, preconditioner diagonal,
  // Dirichlet term, adjoint gradient (three words per value)
  acc_t *g_acc = nullptr, *H_acc = nullptr, *Dc_acc = nullptr, *gdir_acc = nullptr, *gz_acc = nullptr;
  // canonical pair order: sort buffers (up to ow.cap pairs) and the bits of the largest primitive id
  OrderWork ow;
  int prim_bits = 1;
  AbdChunks abd_ch;  // order of the per-body ABD coupling lists
  double *y = nullptr, *partial = nullptr;
  double* T_dev = nullptr;
  // PCG: operator in the CTA-major layout (iteration type), nine iteration vectors, row partition
  double* pcg_op = nullptr;
  double* pcg_vec = nullptr;
  std::vector<int> h_row;      // BSR row offsets (host copy)
  PcgPlan plan;
  int plan_fp32 = -1;
  int* d_seg = nullptr;         // PCG plan: FEM/body segments, ABD CTA ranges, scene of every CTA, CTAs of every scene
  int d_seg_cap = 0;
  std::vector<int> h_plan_buf;  // host staging of d_seg
  std::vector<int> h_node_scene;  // scene of every node (batches)
  int* d_pcg_skip = nullptr;     // (n_scenes) scenes the next PCG leaves out (their Newton iteration has converged)
  int* pcg_skip_h = nullptr;     // pinned staging of d_pcg_skip
  bool pcg_skip_on = false;
  double* d_pcg_sc_res = nullptr;  // (n_scenes) relative residual of every scene's last solve
  bool plan_resident = false;
  size_t plan_smem = 0;
  size_t plan_co_smem = 0;  // shared memory for the coarse rows of every CTA after the plan's (0: none)
  int plan_want_grid = 0, plan_rowg = 0;
  bool pcg_streamed = false;   // never keep the operator in shared memory (sim_pcg_residency)
  bool plan_streamed = false;
  std::vector<int> h_inc_ptr, h_row_extra, plan_row_extra;  // contact-weighted planning (per FEM row)
  // contact incidences per owner (FEM node or ABD body)
  int *inc_ptr = nullptr, *inc_cursor = nullptr, *inc_tiles = nullptr;
  int2* inc = nullptr;
  PairDesc* desc = nullptr;    // (cap + fcap) gather descriptors of the pairs
  long long desc_cap = 0;
  long long inc_cap = 0;
  // contact coupling blocks of the ABD pseudo-node rows
  int *abd_ptr = nullptr, *abd_cursor = nullptr, *abd_ent = nullptr;
  double* abd_val = nullptr;
  float* abd_val32 = nullptr;
  long long abd_cap = 0;
  int* pcg_check = nullptr;    // diagnostic index-check flag of the PCG
  // mixed precision copies
  float *pairH32 = nullptr, *fHu32 = nullptr, *Dinv32 = nullptr;
  // contact
  int cap = 0;
  int* rec = nullptr;
  double* rec_s = nullptr;
  double* pairH = nullptr;
  int ccap = 0;
  int* cand = nullptr;        // contact candidates of the current Newton iteration's sweep
  bool cand_valid = false;
  int fcap = 0, n_fric = 0;
  int* f_ids = nullptr;
  int* f_rec = nullptr;        // (kind, type, primitive a, primitive b) of every friction pair (adjoint)
  double *f_w = nullptr, *f_n = nullptr, *f_lam = nullptr, *f_Hu = nullptr;
  // scalars (device) and pinned host mirror
  struct Scal {
    // cleared at the start of every Newton iteration
    acc_t E[24];                 // 8 accumulators: inertia, elastic, barrier, friction, stitch, abd, joints
                                 // (adjoint scratch: 6, 7)
    unsigned long long pn[2];    // max|p_F|, max|p_D|
    int n_ccd;
    int pcg_out[3];
    int flags;
    int pad;
    double pcg_res;
    // set at the start of every Newton iteration
    unsigned long long alpha;    // CCD bound
    unsigned long long min_s;
    // kept across iterations: sizes of the active-pair and candidate lists
    int n_pairs;
    int n_cand;
  };
  Scal* sc_dev = nullptr;
  Scal* sc_host = nullptr;
  int pcg_grid_max = 1;
  // per-scene Newton control of a batch (n_scenes > 1): device accumulators and pinned host mirrors
  acc_t* E_sc_dev = nullptr;    // (n_scenes, 8) accumulators
  // barrier stiffness per scene (adaptive growth): current, cap, at the start of the step, the smallest
  // squared distance of the previous iterate; device copy of the current values; per-scene minima of a batch
  std::vector<double> kappa_cur, kappa_max, kappa_step, s_prev;
  double* d_scene_kappa = nullptr;
  unsigned long long* min_sc_dev = nullptr;
  std::vector<unsigned long long> min_sc_h;
  double E_h[8] = {0};          // the accumulators of sc_host->E as doubles (sync_scalars)
  std::vector<double> E_sc_v;   // (n_scenes, 8) the same per scene
  // joint drive targets (b-side vectors, offsets), rewritten by sim_set_joint_targets
  int nj = 0;
  double* jt_vb = nullptr;
  double* jt_t = nullptr;
  unsigned long long* alpha_sc_dev = nullptr;
  unsigned long long* pn_sc_dev = nullptr;
  double* alpha_trial_dev = nullptr;
  acc_t* E_sc_h = nullptr;
  unsigned long long* alpha_sc_h = nullptr;
  unsigned long long* pn_sc_h = nullptr;
  // PCG launch shape: threads per FEM row and CTAs per SM
  int tune_rowg = PCG_ROW_GROUP, tune_bps = 2;
  bool autotune_pending = false;
  float tune_ms[8] = {0};
  // optional per-stage CUDA-event timing on the simulator's stream
  bool prof = false;
  cudaEvent_t ev[2 * 8] = {};
  double prof_ms[8] = {0};
  long long prof_n[8] = {0};
  bool ev_open[8] = {false};
  // broad phase
  Bvh tri_tree, edge_tree;
  double bvh_pad = 0;
  // coarse level of the PCG preconditioner (two-level additive Schwarz)
  CoarseLayout co;
  int co_plan_stamp = -1;        // plan_stamp the layout was made for
  int plan_stamp = 0;            // incremented whenever pcg_prepare makes a new plan
  bool co_ok = false;            // the last build succeeded (else block Jacobi only)
  bool co_built_this_step = false;
  int *co_node_agg = nullptr, *co_agg_solve = nullptr, *co_solve_lo = nullptr, *co_solve_n = nullptr;
  int *co_cta_agg = nullptr, *co_agg_cta = nullptr;
  int co_cap_ctas = 0;
  double* co_rot = nullptr;
  // two-level solves repeated with block Jacobi, and the iterations those failed solves took
  long long pcg_fallbacks = 0, pcg_fallback_iters = 0;
  bool co_force_rebuild = false;
  // rebuild policy: the coarse level is kept across steps while the PCG iterations stay near those of
  // the first step after its build
  int co_steps_since_build = 0;
  double co_iters_ref = 0.0;      // PCG iterations per solve in the step of the last build
  long long co_step_iters = 0, co_step_solves = 0;  // this step so far
  double co_last_step_avg = 0.0;  // PCG iterations per solve of the previous step
  int* co_status = nullptr;
  long long *co_off = nullptr, *co_boff = nullptr;
  double *co_Ac = nullptr, *co_centre = nullptr, *co_x = nullptr, *co_part = nullptr, *co_gj = nullptr;
  acc_t* co_Ac_acc = nullptr;
  float* co_Ac32 = nullptr;
  long long co_cap = 0, co_cap_n = 0;
  int co_cap_agg = 0, co_cap_solves = 0;
  std::vector<int> co_status_h;
  // per-step PCG work, for algorithmic-byte accounting
  long long pcg_iters_acc = 0;
  long long pcg_pair_iters_acc = 0;
  long long pcg_fric_iters_acc = 0;
};

namespace {

const int PCG_THREADS = 256;

#define CUDA_TRY(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      sim->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return IPC_ERR_CUDA;                                                    \
    }                                                                         \
  } while (0)

template <typename T>
ipc_status dalloc(ipcsim* sim, T** ptr, size_t count) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = sim->mem.get(&p, bytes);
  if (e != cudaSuccess) {
    sim->err = std::string(sim->mem.alloc_fn ? "device allocator: " : "cudaMalloc: ") + cudaGetErrorString(e) +
               " (" + std::to_string(bytes) + " bytes)";
    return IPC_ERR_CUDA;
  }
  cudaMemsetAsync(p, 0, bytes, sim->st);
  sim->allocs.push_back({p, bytes});
  *ptr = (T*)p;
  return IPC_OK;
}

void dfree(ipcsim* sim, void* p) {
  if (!p) return;
  for (auto it = sim->allocs.begin(); it != sim->allocs.end(); ++it)
    if (it->first == p) {
      // the block may still be read by work queued on the stream: a caching allocator that reuses it
      // for the same stream orders the reuse after that work; cudaFree synchronises
      sim->mem.put(p, it->second);
      sim->allocs.erase(it);
      return;
    }
}

template <typename T>
ipc_status upload(ipcsim* sim, T** ptr, const std::vector<T>& h) {
  ipc_status s = dalloc(sim, ptr, h.size());
  if (s) return s;
  if (!h.empty()) CUDA_TRY(cudaMemcpyAsync(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, sim->st));
  return IPC_OK;
}

// d^2/dd^2 of b(d^2) with kappa = 1: 4 s b''(s) + 2 b'(s), s = d^2
double barrier_dd(double d, double dhat) {
  double sh = dhat * dhat, s = d * d, dd = s - sh, l = std::log(s / sh);
  double b1 = -(2 * dd * l + dd * dd / s);
  double b2 = -(2 * l + 4 * dd / s - dd * dd / (s * s));
  return 4 * s * b2 + 2 * b1;
}

void inv3(const double* m, double* o, double& det) {
  double c00 = m[4] * m[8] - m[5] * m[7], c01 = m[5] * m[6] - m[3] * m[8], c02 = m[3] * m[7] - m[4] * m[6];
  det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  double id = 1.0 / det;
  o[0] = c00 * id; o[1] = (m[2] * m[7] - m[1] * m[8]) * id; o[2] = (m[1] * m[5] - m[2] * m[4]) * id;
  o[3] = c01 * id; o[4] = (m[0] * m[8] - m[2] * m[6]) * id; o[5] = (m[2] * m[3] - m[0] * m[5]) * id;
  o[6] = c02 * id; o[7] = (m[1] * m[6] - m[0] * m[7]) * id; o[8] = (m[0] * m[4] - m[1] * m[3]) * id;
}

// incidence entries: four per barrier pair and per friction pair
ipc_status grow_abd_list(ipcsim* sim, long long need);

ipc_status grow_inc(ipcsim* sim) {
  const long long nd = (long long)sim->cap + sim->fcap;
  if (nd > sim->desc_cap) {
    dfree(sim, sim->desc);
    sim->desc = nullptr;
    ipc_status s = dalloc(sim, &sim->desc, (size_t)nd);
    if (s) return s;
    sim->desc_cap = nd;
  }
  // ABD coupling blocks: twelve per pair cover a pair with one ABD body and three other vertices
  if (sim->nab) {
    ipc_status s = grow_abd_list(sim, 12 * nd);
    if (s) return s;
  }
  long long need = 4LL * ((long long)sim->cap + sim->fcap);
  if (need <= sim->inc_cap) return IPC_OK;
  dfree(sim, sim->inc);
  sim->inc = nullptr;
  ipc_status s = dalloc(sim, &sim->inc, (size_t)need);  // int2 entries
  if (s) return s;
  sim->inc_cap = need;
  return IPC_OK;
}

// Largest pair and candidate buffers the simulator grows to (records of 32 B,
// pair blocks of 1152 B): beyond them a step fails with IPC_ERR_CAPACITY.
constexpr long long MAX_PAIRS = 1LL << 23;
constexpr long long MAX_CANDIDATES = 1LL << 26;
// the pair buffer limit of this simulator: pair_capacity_max when set, else MAX_PAIRS
long long max_pairs(const ipcsim* sim) {
  return sim->P.pair_capacity_max > 0 ? std::min<long long>(sim->P.pair_capacity_max, MAX_PAIRS) : MAX_PAIRS;
}

// ABD coupling blocks: a few per pair touching an ABD body; grown when a Newton iteration overflows them
ipc_status grow_abd_list(ipcsim* sim, long long need) {
  if (sim->nab == 0 || need <= sim->abd_cap) return IPC_OK;
  if (need > (1LL << 30)) { sim->err = "ABD coupling list exceeds 2^30 entries"; return IPC_ERR_CAPACITY; }
  AbdChunks& C = sim->abd_ch;
  for (void* p : {(void*)sim->abd_ent, (void*)sim->abd_val, (void*)sim->abd_val32, (void*)C.ent_raw, (void*)C.val_raw,
                  (void*)C.ekeys, (void*)C.ekeys_tmp, (void*)C.eidx, (void*)C.eidx_tmp, (void*)C.ehist,
                  (void*)C.etiles, (void*)C.ehead, (void*)C.body_cnt})
    dfree(sim, p);
  sim->abd_ent = nullptr;
  sim->abd_val = nullptr;
  sim->abd_val32 = nullptr;
  C.ent_raw = nullptr; C.val_raw = nullptr; C.ekeys = nullptr; C.ekeys_tmp = nullptr; C.eidx = nullptr;
  C.eidx_tmp = nullptr; C.ehist = nullptr; C.etiles = nullptr; C.ehead = nullptr; C.body_cnt = nullptr;
  ipc_status s;
  const size_t n = (size_t)need, nh = sort_hist_ints((int)need);
  if ((s = dalloc(sim, &sim->abd_ent, n))) return s;
  if ((s = dalloc(sim, &sim->abd_val, 9 * n))) return s;
  if (sim->P.precision == IPC_PREC_MIXED && (s = dalloc(sim, &sim->abd_val32, 9 * n))) return s;
  if ((s = dalloc(sim, &C.ent_raw, n)) || (s = dalloc(sim, &C.val_raw, 9 * n)) || (s = dalloc(sim, &C.ekeys, n)) ||
      (s = dalloc(sim, &C.ekeys_tmp, n)) || (s = dalloc(sim, &C.eidx, n)) || (s = dalloc(sim, &C.eidx_tmp, n)) ||
      (s = dalloc(sim, &C.ehist, nh)) || (s = dalloc(sim, &C.etiles, std::max(scan_tile_ints(nh), scan_tile_ints(n)))) ||
      (s = dalloc(sim, &C.ehead, n)) || (s = dalloc(sim, &C.body_cnt, (size_t)sim->nab + 1)))
    return s;
  C.code_bits = 3;
  while ((1LL << (C.code_bits - 2)) <= sim->n_nodes) ++C.code_bits;
  int body_bits = 1;
  while ((1LL << body_bits) <= sim->nab) ++body_bits;
  C.ekey_bits = body_bits + C.code_bits;
  C.ecap = need;
  sim->abd_cap = need;
  return IPC_OK;
}

// Sort buffers for pair lists of up to cap entries.
ipc_status grow_order(ipcsim* sim, int cap) {
  OrderWork& W = sim->ow;
  if (cap <= W.cap) return IPC_OK;
  dfree(sim, W.keys); dfree(sim, W.keys_tmp); dfree(sim, W.idx); dfree(sim, W.idx_tmp); dfree(sim, W.hist);
  dfree(sim, W.tiles); dfree(sim, W.rec_tmp); dfree(sim, W.s_tmp);
  W = OrderWork{};
  ipc_status s;
  const size_t nh = sort_hist_ints(cap);
  if ((s = dalloc(sim, &W.keys, (size_t)cap)) || (s = dalloc(sim, &W.keys_tmp, (size_t)cap)) ||
      (s = dalloc(sim, &W.idx, (size_t)cap)) || (s = dalloc(sim, &W.idx_tmp, (size_t)cap)) ||
      (s = dalloc(sim, &W.hist, nh)) || (s = dalloc(sim, &W.tiles, scan_tile_ints(nh))) ||
      (s = dalloc(sim, &W.rec_tmp, 8 * (size_t)cap)) || (s = dalloc(sim, &W.s_tmp, (size_t)cap)))
    return s;
  W.cap = cap;
  return IPC_OK;
}

ipc_status grow_pairs(ipcsim* sim, int need) {
  const long long lim = max_pairs(sim);
  if (need < 0 || need > lim) {
    sim->err = "active-pair count " + std::to_string(need) + " exceeds the pair buffer limit " + std::to_string(lim);
    return IPC_ERR_CAPACITY;
  }
  int ncap = (int)std::min<long long>(std::max<long long>(need + (long long)need / 2, 1024), lim);
  dfree(sim, sim->rec);
  dfree(sim, sim->rec_s);
  dfree(sim, sim->pairH);
  sim->rec = nullptr; sim->rec_s = nullptr; sim->pairH = nullptr;
  ipc_status s;
  if ((s = dalloc(sim, &sim->rec, (size_t)8 * ncap))) return s;
  if ((s = dalloc(sim, &sim->rec_s, (size_t)ncap))) return s;
  if ((s = dalloc(sim, &sim->pairH, (size_t)144 * ncap))) return s;
  if (sim->P.precision == IPC_PREC_MIXED) {
    dfree(sim, sim->pairH32);
    sim->pairH32 = nullptr;
    if ((s = dalloc(sim, &sim->pairH32, (size_t)144 * ncap))) return s;
  }
  sim->cap = ncap;
  if ((s = grow_order(sim, ncap))) return s;
  return grow_inc(sim);
}

ipc_status grow_cand(ipcsim* sim, int need) {
  if (need < 0 || need > MAX_CANDIDATES) {
    sim->err = "CCD candidate count " + std::to_string(need) + " exceeds the candidate buffer limit";
    return IPC_ERR_CAPACITY;
  }
  int ncap = (int)std::min<long long>(std::max<long long>(need + (long long)need / 2, 4096), MAX_CANDIDATES);
  dfree(sim, sim->cand);
  sim->cand = nullptr;
  ipc_status s = dalloc(sim, &sim->cand, (size_t)8 * ncap);
  if (s) return s;
  sim->ccap = ncap;
  sim->cand_valid = false;
  return IPC_OK;
}

ipc_status grow_fric(ipcsim* sim, int need) {
  const long long lim = max_pairs(sim);
  if (need < 0 || need > lim) {
    sim->err = "friction-pair count " + std::to_string(need) + " exceeds the pair buffer limit " + std::to_string(lim);
    return IPC_ERR_CAPACITY;
  }
  int ncap = (int)std::min<long long>(std::max<long long>(need + (long long)need / 2, 1024), lim);
  dfree(sim, sim->f_ids); dfree(sim, sim->f_w); dfree(sim, sim->f_n); dfree(sim, sim->f_lam); dfree(sim, sim->f_Hu);
  dfree(sim, sim->f_rec);
  ipc_status s;
  if ((s = dalloc(sim, &sim->f_ids, (size_t)4 * ncap))) return s;
  if ((s = dalloc(sim, &sim->f_rec, (size_t)4 * ncap))) return s;
  if ((s = dalloc(sim, &sim->f_w, (size_t)4 * ncap))) return s;
  if ((s = dalloc(sim, &sim->f_n, (size_t)3 * ncap))) return s;
  if ((s = dalloc(sim, &sim->f_lam, (size_t)ncap))) return s;
  if ((s = dalloc(sim, &sim->f_Hu, (size_t)9 * ncap))) return s;
  if (sim->P.precision == IPC_PREC_MIXED) {
    dfree(sim, sim->fHu32);
    sim->fHu32 = nullptr;
    if ((s = dalloc(sim, &sim->fHu32, (size_t)9 * ncap))) return s;
  }
  sim->fcap = ncap;
  return grow_inc(sim);
}

enum { PROF_PCG = 0, PROF_ELASTIC = 1, PROF_BARRIER = 2, PROF_CULL = 3, PROF_CCD = 4, PROF_FRICTION = 5,
       PROF_OTHER = 6, PROF_PCG_SETUP = 7 };

inline void prof_begin(ipcsim* sim, int k) {
  if (!sim->prof) return;
  if (!sim->ev[2 * k]) {
    cudaEventCreate(&sim->ev[2 * k]);
    cudaEventCreate(&sim->ev[2 * k + 1]);
  }
  cudaEventRecord(sim->ev[2 * k], sim->st);
}
inline void prof_end(ipcsim* sim, int k) {
  if (!sim->prof) return;
  cudaEventRecord(sim->ev[2 * k + 1], sim->st);
  sim->ev_open[k] = true;
}
// called after a stream synchronisation: accumulate the recorded intervals
inline void prof_collect(ipcsim* sim) {
  if (!sim->prof) return;
  for (int k = 0; k < 8; ++k)
    if (sim->ev_open[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, sim->ev[2 * k], sim->ev[2 * k + 1]) == cudaSuccess) {
        sim->prof_ms[k] += ms;
        sim->prof_n[k] += 1;
      }
      sim->ev_open[k] = false;
    }
}

// Row partition, shared-memory residency and operator layout of the PCG for
// the current launch shape (tune_rowg threads per FEM row, tune_bps CTAs per SM).
// Plan of the cooperative PCG launch and the operator layout of the current Hessian.  With
// contacts = true the FEM rows are re-partitioned with the contact work of the current incidence lists
// (PCG_CONTACT_WEIGHT per incidence, in units of a BSR block) when it changed; otherwise the plan is kept.
ipc_status pcg_prepare(ipcsim* sim, int fp32, bool contacts = false) {
  const int sms = device_sms();
  const int rowg = sim->tune_rowg;
  const int want = std::min(std::max(1, sms * std::max(1, sim->tune_bps)), sim->pcg_grid_max);
  const int contact_w = PCG_CONTACT_WEIGHT;
  bool extra_changed = false;
  if (contacts && contact_w > 0 && sim->nf > 0) {
    sim->h_inc_ptr.resize(sim->nf + 1);
    CUDA_TRY(cudaMemcpyAsync(sim->h_inc_ptr.data(), sim->inc_ptr, sizeof(int) * (sim->nf + 1), cudaMemcpyDeviceToHost,
                             sim->st));
    CUDA_TRY(cudaStreamSynchronize(sim->st));
    sim->h_row_extra.resize(sim->nf);
    for (int i = 0; i < sim->nf; ++i) sim->h_row_extra[i] = contact_w * (sim->h_inc_ptr[i + 1] - sim->h_inc_ptr[i]);
    extra_changed = sim->h_row_extra != sim->plan_row_extra;
  }
  if (extra_changed ||
      !(sim->plan.grid > 0 && sim->plan_want_grid == want && sim->plan_fp32 == fp32 && sim->plan_rowg == rowg &&
        sim->plan_streamed == sim->pcg_streamed)) {
    // shrink the grid until every CTA of the plan is co-resident, re-planning the rows for every grid
    // size (fewer CTAs own more rows each, which can need more shared memory)
    int grid = want;
    bool resident = false, fits = false;
    size_t smem = 0;
    for (int attempt = 0; attempt < 32 && !fits; ++attempt) {
      if (grid < 1 || (sim->nab > 0 && grid < 2)) break;
      pcg_plan_rows(sim->h_row, sim->nf, sim->nab, grid, sim->h_node_scene, sim->n_scenes, sim->plan,
                    sim->h_row_extra.empty() ? nullptr : &sim->h_row_extra);
      const size_t bytes = pcg_resident_bytes(sim->plan, fp32);
      const int cap_res = (!sim->pcg_streamed && bytes <= pcg_smem_limit()) ? pcg_max_blocks(PCG_THREADS, fp32, rowg, bytes) : 0;
      if (cap_res >= grid) { resident = true; smem = bytes; fits = true; break; }
      smem = pcg_contact_bytes(sim->plan);
      const int cap = smem <= pcg_smem_limit() ? pcg_max_blocks(PCG_THREADS, fp32, rowg, smem) : 0;
      if (cap < grid && !sim->h_row_extra.empty()) {
        // the contact-weighted partition gave a CTA more rows than this grid's shared memory per CTA holds
        // (cheap rows gather in few CTAs): plan this grid without the contact work before shrinking it
        sim->h_row_extra.clear();
        --attempt;
        continue;
      }
      if (cap <= 0) {
        sim->err = "PCG kernel cannot be made resident (grid " + std::to_string(grid) + ", largest segment " +
                   std::to_string(sim->plan.max_rows) + " rows, " + std::to_string(smem) + " B of shared memory)";
        return IPC_ERR_CUDA;
      }
      if (cap >= grid) { fits = true; break; }
      grid = cap;
    }
    if (!fits) {
      sim->err = "no PCG launch shape with every CTA co-resident (grid " + std::to_string(grid) + ")";
      return IPC_ERR_CUDA;
    }
    // one device buffer: seg | abd_seg | cta_scene | sc_ptr | sc_cta
    const PcgPlan& pl = sim->plan;
    std::vector<int>& buf = sim->h_plan_buf;
    CUDA_TRY(cudaStreamSynchronize(sim->st));  // the previous upload from buf has completed
    buf.clear();
    for (const std::vector<int>* v : {&pl.seg, &pl.abd_seg, &pl.cta_scene, &pl.sc_ptr, &pl.sc_cta})
      buf.insert(buf.end(), v->begin(), v->end());
    const int n = (int)buf.size();
    if (n > sim->d_seg_cap) {
      dfree(sim, sim->d_seg);
      sim->d_seg = nullptr;
      ipc_status s = dalloc(sim, &sim->d_seg, (size_t)n);
      if (s) return s;
      sim->d_seg_cap = n;
    }
    CUDA_TRY(cudaMemcpyAsync(sim->d_seg, buf.data(), sizeof(int) * n, cudaMemcpyHostToDevice, sim->st));
    sim->plan_want_grid = want;
    sim->plan_row_extra = sim->h_row_extra;
    sim->plan_fp32 = fp32;
    sim->plan_rowg = rowg;
    sim->plan_streamed = sim->pcg_streamed;
    sim->plan_resident = resident;
    sim->plan_smem = smem;
    // room for the six coarse rows of every CTA (one solve's largest coarse size) when it keeps the grid
    sim->plan_co_smem = 0;
    if (sim->P.preconditioner == IPC_PRECOND_TWO_LEVEL && sim->nf > 0) {
      const size_t co = 6 * (size_t)COARSE_MAX_UNKNOWNS * (fp32 ? sizeof(float) : sizeof(double));
      if (smem + co <= pcg_smem_limit() && pcg_max_blocks(PCG_THREADS, fp32, rowg, smem + co) >= sim->plan.grid)
        sim->plan_co_smem = co;
    }
    ++sim->plan_stamp;
  }
  launch_layout(sim->st, sim->plan.n_fem_ctas + sim->nab, sim->d_seg, sim->S.bsr_row, sim->Hval, sim->pcg_op,
                fp32);
  return IPC_OK;
}

// Coarse level of the preconditioner for the current plan and assembled system
// (Hval, pair and friction blocks): the layout (again when the plan changed),
// the rigid-body modes at the current FEM positions xv, the Galerkin matrix
// P^T A P of every solve and its inverse.  On a failed inversion the PCG runs
// with block Jacobi alone (co_ok false).
ipc_status coarse_setup(ipcsim* sim, int fp32, int n_fric) {
  sim->co_ok = false;
  sim->co_force_rebuild = false;
  if (sim->P.preconditioner != IPC_PRECOND_TWO_LEVEL || sim->nf == 0 || sim->plan.n_fem_ctas <= 0) return IPC_OK;
  CoarseLayout& L = sim->co;
  if (sim->co_plan_stamp != sim->plan_stamp) {
    coarse_layout(sim->plan, sim->nf, L);
    sim->co_plan_stamp = sim->plan_stamp;
    if (!L.consecutive || L.total <= 0) return IPC_OK;
    ipc_status s;
    if (L.total > sim->co_cap) {
      dfree(sim, sim->co_Ac); dfree(sim, sim->co_Ac32); dfree(sim, sim->co_Ac_acc);
      sim->co_Ac = nullptr; sim->co_Ac32 = nullptr; sim->co_Ac_acc = nullptr;
      if ((s = dalloc(sim, &sim->co_Ac, (size_t)L.total))) return s;
      if ((s = dalloc(sim, &sim->co_Ac_acc, 3 * (size_t)L.total))) return s;
      if ((s = dalloc(sim, &sim->co_Ac32, (size_t)L.total))) return s;
      sim->co_cap = L.total;
    }
    if (L.n_ctas > sim->co_cap_ctas) {
      dfree(sim, sim->co_cta_agg); dfree(sim, sim->co_part);
      sim->co_cta_agg = nullptr; sim->co_part = nullptr;
      if ((s = dalloc(sim, &sim->co_cta_agg, (size_t)L.n_ctas))) return s;
      if ((s = dalloc(sim, &sim->co_part, 6 * (size_t)L.n_ctas))) return s;
      sim->co_cap_ctas = L.n_ctas;
    }
    if (L.total_n > sim->co_cap_n) {
      dfree(sim, sim->co_gj);
      sim->co_gj = nullptr;
      if ((s = dalloc(sim, &sim->co_gj, 4 * (size_t)L.total_n))) return s;
      sim->co_cap_n = L.total_n;
    }
    if (L.n_agg > sim->co_cap_agg) {
      dfree(sim, sim->co_agg_solve); dfree(sim, sim->co_centre); dfree(sim, sim->co_rot); dfree(sim, sim->co_agg_cta);
      sim->co_agg_solve = nullptr; sim->co_centre = nullptr; sim->co_rot = nullptr; sim->co_agg_cta = nullptr;
      if ((s = dalloc(sim, &sim->co_agg_solve, (size_t)L.n_agg))) return s;
      if ((s = dalloc(sim, &sim->co_centre, 3 * (size_t)L.n_agg))) return s;
      if ((s = dalloc(sim, &sim->co_rot, (size_t)L.n_agg))) return s;
      if ((s = dalloc(sim, &sim->co_agg_cta, 2 * (size_t)L.n_agg + 1))) return s;
      sim->co_cap_agg = L.n_agg;
    }
    if (L.n_solves > sim->co_cap_solves) {
      dfree(sim, sim->co_solve_lo); dfree(sim, sim->co_solve_n); dfree(sim, sim->co_off); dfree(sim, sim->co_boff);
      dfree(sim, sim->co_status);
      sim->co_solve_lo = nullptr; sim->co_solve_n = nullptr; sim->co_off = nullptr; sim->co_boff = nullptr;
      sim->co_status = nullptr;
      if ((s = dalloc(sim, &sim->co_solve_lo, (size_t)L.n_solves))) return s;
      if ((s = dalloc(sim, &sim->co_solve_n, (size_t)L.n_solves))) return s;
      if ((s = dalloc(sim, &sim->co_off, (size_t)L.n_solves))) return s;
      if ((s = dalloc(sim, &sim->co_boff, (size_t)L.n_solves))) return s;
      if ((s = dalloc(sim, &sim->co_status, (size_t)L.n_solves))) return s;
      sim->co_cap_solves = L.n_solves;
    }
    if (!sim->co_node_agg && (s = dalloc(sim, &sim->co_node_agg, (size_t)sim->nf))) return s;
    if (!sim->co_x && (s = dalloc(sim, &sim->co_x, 3 * (size_t)sim->nf))) return s;
    cudaStream_t cs = sim->st;
    CUDA_TRY(cudaMemcpyAsync(sim->co_node_agg, L.node_agg.data(), sizeof(int) * sim->nf, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_agg_solve, L.agg_solve.data(), sizeof(int) * L.n_agg, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_cta_agg, L.cta_agg.data(), sizeof(int) * L.n_ctas, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_agg_cta, L.agg_cta.data(), sizeof(int) * L.agg_cta.size(), cudaMemcpyHostToDevice,
                             cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_solve_lo, L.solve_lo.data(), sizeof(int) * L.n_solves, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_solve_n, L.solve_n.data(), sizeof(int) * L.n_solves, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_off, L.off.data(), sizeof(long long) * L.n_solves, cudaMemcpyHostToDevice, cs));
    CUDA_TRY(cudaMemcpyAsync(sim->co_boff, L.boff.data(), sizeof(long long) * L.n_solves, cudaMemcpyHostToDevice, cs));
    // the host vectors are read by the copies: wait for them before they can change
    CUDA_TRY(cudaStreamSynchronize(cs));
  }
  if (!L.consecutive || L.total <= 0) return IPC_OK;
  cudaStream_t cs = sim->st;
  CUDA_TRY(cudaMemcpyAsync(sim->co_x, sim->xv, sizeof(double) * 3 * sim->nf, cudaMemcpyDeviceToDevice, cs));
  CUDA_TRY(cudaMemsetAsync(sim->co_part, 0, sizeof(double) * 6 * L.n_ctas, cs));
  CoarseDevLayout D;
  D.n_agg = L.n_agg; D.n_solves = L.n_solves; D.n_max = L.n_max; D.total = L.total; D.total_n = L.total_n;
  D.node_agg = sim->co_node_agg; D.agg_solve = sim->co_agg_solve; D.solve_lo = sim->co_solve_lo;
  D.solve_n = sim->co_solve_n; D.off = sim->co_off; D.boff = sim->co_boff; D.agg_cta = sim->co_agg_cta;
  CUDA_TRY(launch_coarse_build(cs, sim->S, D, sim->d_seg, sim->co_x, sim->Hval, sim->rec, &sim->sc_dev->n_pairs,
                               sim->cap, sim->pairH, n_fric, sim->f_ids, sim->f_w, sim->f_Hu, sim->co_Ac,
                               sim->co_Ac_acc, sim->co_centre, sim->co_rot, sim->co_gj, sim->co_status));
  sim->co_status_h.assign(L.n_solves, 0);
  CUDA_TRY(cudaMemcpyAsync(sim->co_status_h.data(), sim->co_status, sizeof(int) * L.n_solves, cudaMemcpyDeviceToHost,
                           cs));
  CUDA_TRY(cudaStreamSynchronize(cs));
  for (int v : sim->co_status_h)
    if (v) return IPC_OK;  // a pivot failed: block Jacobi alone for this build
  launch_to_float(cs, (size_t)L.total, sim->co_Ac, sim->co_Ac32);
  sim->co_ok = true;
  return IPC_OK;
}

// One PCG solve of H_FF p = rhs on the assembled system (Hval, pairH, f_Hu,
// Dinv and, for FP32 iterations, their FP32 copies); the incidence lists
// must describe the current pairs and pcg_prepare must have run on this Hval.
ipc_status pcg_launch(ipcsim* sim, int fp32, double rtol, int max_iter, int n_fric, bool use_coarse);

// One linear solve.  A two-level solve that broke down or ended far above its tolerance (the coarse
// inverse was not positive definite on this system) is repeated with block Jacobi alone, and the coarse
// level is rebuilt at the next Newton iteration; fallbacks and the iterations of the failed solves are
// counted in sim->pcg_fallbacks / sim->pcg_fallback_iters.
ipc_status pcg_run(ipcsim* sim, int fp32, double rtol, int max_iter, int n_fric) {
  ipc_status s = pcg_launch(sim, fp32, rtol, max_iter, n_fric, true);
  if (s || !sim->co_ok) return s;
  ipcsim::Scal* h = sim->sc_host;
  CUDA_TRY(cudaMemcpyAsync(h->pcg_out, sim->sc_dev->pcg_out, sizeof(h->pcg_out), cudaMemcpyDeviceToHost, sim->st));
  CUDA_TRY(cudaMemcpyAsync(&h->pcg_res, &sim->sc_dev->pcg_res, sizeof(double), cudaMemcpyDeviceToHost, sim->st));
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  const int status = h->pcg_out[1];
  if (status == 1 || status == 2 || (status == 3 && !(h->pcg_res < 0.5))) {
    ++sim->pcg_fallbacks;
    sim->pcg_fallback_iters += h->pcg_out[0];
    sim->co_force_rebuild = true;
    return pcg_launch(sim, fp32, rtol, max_iter, n_fric, false);
  }
  return IPC_OK;
}

ipc_status pcg_launch(ipcsim* sim, int fp32, double rtol, int max_iter, int n_fric, bool use_coarse) {
  const DevScene& S = sim->S;
  PcgArgs a{};
  a.S = S;
  a.n_nodes = sim->n_nodes;
  a.n_fem_ctas = sim->plan.n_fem_ctas;
  a.n_abd_ctas = sim->plan.n_abd_ctas;
  a.seg_row = sim->d_seg;
  {
    const PcgPlan& pl = sim->plan;
    const int* d = sim->d_seg + pl.seg.size();
    a.abd_seg = d; d += pl.abd_seg.size();
    a.cta_scene = d; d += pl.cta_scene.size();
    a.sc_ptr = d; d += pl.sc_ptr.size();
    a.sc_cta = d;
    a.n_psc = pl.n_psc;
    // the per-scene plan's solves are the scenes of the batch
    const bool per_scene = pl.n_psc > 1 && pl.n_psc == sim->n_scenes;
    a.scene_skip = per_scene && sim->pcg_skip_on ? sim->d_pcg_skip : nullptr;
    a.sc_res = per_scene ? sim->d_pcg_sc_res : nullptr;
    a.sc_it = nullptr;
  }
  a.resident = sim->plan_resident ? 1 : 0;
  a.row = S.bsr_row;
  a.col = S.bsr_col;
  a.op = sim->pcg_op;
  a.dinv = fp32 ? (const void*)sim->Dinv32 : (const void*)sim->Dinv;
  a.val64 = sim->Hval;
  a.pairH = fp32 ? (const void*)sim->pairH32 : (const void*)sim->pairH;
  a.fHu = fp32 ? (const void*)sim->fHu32 : (const void*)sim->f_Hu;
  a.pairH64 = sim->pairH;
  a.fHu64 = sim->f_Hu;
  a.rec = sim->rec;
  a.n_pairs = &sim->sc_dev->n_pairs;
  a.cap = sim->cap;
  a.n_fric = n_fric;
  a.f_ids = sim->f_ids;
  a.f_w = sim->f_w;
  a.desc = sim->desc;
  a.inc_ptr = sim->inc_ptr;
  a.inc = sim->inc;
  a.b = sim->rhs;
  a.x = sim->p;
  a.vec = sim->pcg_vec;
  a.t64 = sim->y;
  a.partial = sim->partial;
  a.rtol = rtol;
  a.max_iter = max_iter;
  a.max_replace = sim->pcg_max_replace;
  a.fp32 = fp32;
  a.out = sim->sc_dev->pcg_out;
  a.res = &sim->sc_dev->pcg_res;
  a.inc_cap = sim->inc_cap;
  // IPCSIM_PCG_CHECK=1: the solver validates every gathered index (diagnostic mode)
  static const bool check = [] { const char* e = std::getenv("IPCSIM_PCG_CHECK"); return e && e[0] == '1'; }();
  if (check && !sim->pcg_check) {
    ipc_status s = dalloc(sim, &sim->pcg_check, 1);
    if (s) return s;
  }
  a.check = check ? sim->pcg_check : nullptr;
  a.max_rows = sim->plan.max_rows;
  a.acc_doubles = sim->plan.acc_doubles;
  a.abd_ptr = sim->abd_ptr;
  a.abd_ent = sim->abd_ent;
  a.abd_val = sim->abd_val;
  a.abd_val32 = sim->abd_val32;
  a.abd_cap = sim->abd_cap;
  if (sim->co_ok && use_coarse) {
    a.co.inv32 = sim->co_Ac32;
    // the FP64 (pipelined) solver needs a fixed, symmetric linear preconditioner: it applies the coarse
    // inverse in FP64 (with the FP32 product its recurrences lost r^T M^-1 r > 0 in a third of the grasp's
    // solves); the mixed solver's FP32 inner iteration uses the FP32 copy
    a.co.inv64 = !fp32 ? sim->co_Ac : nullptr;
    a.co.cta_agg = sim->co_cta_agg;
    a.co.agg_cta = sim->co_agg_cta;
    a.co.off = sim->co_off;
    a.co.solve_lo = sim->co_solve_lo;
    a.co.solve_n = sim->co_solve_n;
    a.co.centre = sim->co_centre;
    a.co.rot = sim->co_rot;
    a.co.x = sim->co_x;
    a.co.part = sim->co_part;
  }
  a.co.smem_off = (a.co.inv32 && sim->plan_co_smem) ? (int)sim->plan_smem : -1;
  CUDA_TRY(launch_pcg(sim->st, sim->plan.grid, PCG_THREADS, a, sim->tune_rowg,
                      sim->plan_smem + (a.co.smem_off >= 0 ? sim->plan_co_smem : 0)));
  if (check) {
    int site = 0;
    CUDA_TRY(cudaMemcpyAsync(&site, sim->pcg_check, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
    CUDA_TRY(cudaStreamSynchronize(sim->st));
    if (site) {
      sim->err = "PCG index check failed at site " + std::to_string(site);
      return IPC_ERR_CUDA;
    }
  }
  return IPC_OK;
}

// Chunk-order buffers of the ABD coupling lists for 4 (cap + n_fric) chunk slots.
ipc_status grow_abd_chunks(ipcsim* sim, int n_fric) {
  AbdChunks& C = sim->abd_ch;
  const long long need = 4LL * ((long long)sim->cap + n_fric);
  if (need <= C.cap) return IPC_OK;
  if (need > (1LL << 30)) { sim->err = "ABD coupling chunk count exceeds 2^30"; return IPC_ERR_CAPACITY; }
  for (void* p : {(void*)C.keys, (void*)C.keys_tmp, (void*)C.idx, (void*)C.idx_tmp, (void*)C.hist, (void*)C.tiles,
                  (void*)C.size, (void*)C.scan, (void*)C.pos, (void*)C.n})
    dfree(sim, p);
  // the chunk buffers only: the raw lists and merge buffers (grow_abd_list) stay
  C.keys = C.keys_tmp = nullptr;
  C.idx = C.idx_tmp = C.hist = C.tiles = C.size = C.scan = C.pos = C.n = nullptr;
  C.cap = 0;
  const int cap = (int)std::min<long long>(need + need / 2, 1LL << 30);
  const size_t nh = sort_hist_ints(cap);
  ipc_status s;
  if ((s = dalloc(sim, &C.keys, (size_t)cap)) || (s = dalloc(sim, &C.keys_tmp, (size_t)cap)) ||
      (s = dalloc(sim, &C.idx, (size_t)cap)) || (s = dalloc(sim, &C.idx_tmp, (size_t)cap)) ||
      (s = dalloc(sim, &C.hist, nh)) || (s = dalloc(sim, &C.tiles, std::max(scan_tile_ints(nh), scan_tile_ints(cap)))) ||
      (s = dalloc(sim, &C.size, (size_t)cap)) || (s = dalloc(sim, &C.scan, (size_t)cap)) ||
      (s = dalloc(sim, &C.pos, (size_t)cap)) || (s = dalloc(sim, &C.n, 1)))
    return s;
  C.cap = cap;
  C.pair_bits = 1;
  while ((1LL << C.pair_bits) <= cap / 4) ++C.pair_bits;
  int body_bits = 1;
  while ((1LL << body_bits) <= sim->nab) ++body_bits;
  C.key_bits = body_bits + C.pair_bits + 2;
  return IPC_OK;
}

// ABD contact: same-body blocks into the BSR grid, coupling blocks into the per-body lists.
ipc_status build_abd_contact(ipcsim* sim, int n_fric) {
  if (!sim->nab) return IPC_OK;
  ipc_status s = grow_abd_chunks(sim, n_fric);
  if (s) return s;
  launch_abd_contact(sim->st, sim->S, sim->rec, &sim->sc_dev->n_pairs, sim->cap, sim->pairH, n_fric, sim->f_ids,
                     sim->f_w, sim->f_Hu, sim->abd_ptr, sim->abd_ch, sim->abd_ent, sim->abd_val, sim->abd_cap,
                     sim->H_acc, sim->Dc_acc, &sim->sc_dev->flags);
  return IPC_OK;
}

// Contact incidences of the current pairs (and friction pairs) per owner.
void build_incidence(ipcsim* sim, int n_fric) {
  launch_incidence(sim->st, sim->S, sim->rec, &sim->sc_dev->n_pairs, sim->cap, n_fric, sim->f_ids, sim->f_w,
                   sim->inc_ptr, sim->inc_cursor, sim->inc_tiles, sim->inc, sim->inc_cap, sim->desc,
                   &sim->sc_dev->flags);
}

int pair_grid(int cap) { return stride_grid(cap, 128, 8); }

unsigned long long double_bits(double d);
double bits_to_double(unsigned long long b);

// Cull the active set at xv into sim->rec; count into sc_dev->n_pairs.
void cull_into(ipcsim* sim, const double* xv, int* rec, double* rec_s, int cap) {
  cudaMemsetAsync(&sim->sc_dev->n_pairs, 0, sizeof(int), sim->st);
  if (sim->P.broad_phase == IPC_BROAD_ALL_PAIRS)
    launch_cull_brute(sim->st, sim->S, xv, sim->sh, rec, rec_s, &sim->sc_dev->n_pairs, cap);
  else
    launch_cull_bvh(sim->st, sim->S, xv, sim->sh, sim->bvh_pad, sim->tri_tree, sim->edge_tree, rec, rec_s,
                    &sim->sc_dev->n_pairs, cap, &sim->sc_dev->flags);
  // canonical (kind, a, b) order (the sort buffers cover cap: grown with the pair buffer, or by the caller)
  launch_sort_pairs(sim->st, &sim->sc_dev->n_pairs, std::min(cap, sim->ow.cap), sim->prim_bits, rec, rec_s, sim->ow);
}
void cull(ipcsim* sim, const double* xv) { cull_into(sim, xv, sim->rec, sim->rec_s, sim->cap); }

// Active set at xv: from the current sweep's candidates when they cover xv, else a full cull.
void active_set(ipcsim* sim, const double* xv) {
  if (sim->cand_valid) {
    cudaMemsetAsync(&sim->sc_dev->n_pairs, 0, sizeof(int), sim->st);
    launch_filter_active(sim->st, stride_grid(sim->ccap, 128, 8), sim->S, xv, sim->sh,
                         sim->cand, &sim->sc_dev->n_cand, sim->ccap, sim->rec, sim->rec_s, &sim->sc_dev->n_pairs,
                         sim->cap);
    launch_sort_pairs(sim->st, &sim->sc_dev->n_pairs, sim->cap, sim->prim_bits, sim->rec, sim->rec_s, sim->ow);
  } else {
    cull(sim, xv);
  }
}

// Clear the accumulators of one assembly (gradient, BSR values, preconditioner diagonal, Dirichlet term).
// The FEM blocks are written whole by the elastic assembly; only the ABD blocks accumulate.
ipc_status assembly_begin(ipcsim* sim) {
  const size_t ndof = 3 * (size_t)sim->n_nodes;
  CUDA_TRY(cudaMemsetAsync(sim->g_acc, 0, sizeof(acc_t) * 3 * ndof, sim->st));
  CUDA_TRY(cudaMemsetAsync(sim->H_acc + 27 * (size_t)sim->nfb, 0, sizeof(acc_t) * 27 * (size_t)(sim->nnzb - sim->nfb),
                           sim->st));
  CUDA_TRY(cudaMemsetAsync(sim->Dc_acc, 0, sizeof(acc_t) * 27 * (size_t)sim->n_nodes, sim->st));
  CUDA_TRY(cudaMemsetAsync(sim->gdir_acc, 0, sizeof(acc_t) * 3 * ndof, sim->st));
  return IPC_OK;
}

// The assembled values: g, the ABD blocks Hval = Hconst + the accumulated Hessian terms, Dc, gdir.
void assembly_end(ipcsim* sim) {
  const size_t ndof = 3 * (size_t)sim->n_nodes, f = 9 * (size_t)sim->nfb;
  launch_acc_finalize(sim->st, ndof, sim->g_acc, nullptr, sim->g);
  launch_acc_finalize(sim->st, 9 * (size_t)sim->nnzb - f, sim->H_acc + 3 * f, sim->Hconst + f, sim->Hval + f);
  launch_acc_finalize(sim->st, 9 * (size_t)sim->n_nodes, sim->Dc_acc, nullptr, sim->Dc);
  launch_acc_finalize(sim->st, ndof, sim->gdir_acc, nullptr, sim->gdir);
}

// Clear the per-iteration scalars and set the CCD bound and minimum distance to their neutral values.
ipc_status reset_iteration_scalars(ipcsim* sim) {
  CUDA_TRY(cudaMemsetAsync(sim->sc_dev, 0, offsetof(ipcsim::Scal, alpha), sim->st));
  unsigned long long init[2] = {double_bits(1.0), double_bits(1e300)};
  CUDA_TRY(cudaMemcpyAsync(&sim->sc_dev->alpha, init, sizeof(init), cudaMemcpyHostToDevice, sim->st));
  if (sim->n_scenes > 1) {
    const int ns = sim->n_scenes;
    CUDA_TRY(cudaMemsetAsync(sim->E_sc_dev, 0, sizeof(acc_t) * 24 * ns, sim->st));
    CUDA_TRY(cudaMemsetAsync(sim->pn_sc_dev, 0, sizeof(unsigned long long) * 2 * ns, sim->st));
    // 0x7f bytes: a double near 1.4e306, above every squared distance
    CUDA_TRY(cudaMemsetAsync(sim->min_sc_dev, 0x7f, sizeof(unsigned long long) * ns, sim->st));
    for (int k = 0; k < ns; ++k) sim->alpha_sc_h[k] = double_bits(1.0);
    CUDA_TRY(cudaMemcpyAsync(sim->alpha_sc_dev, sim->alpha_sc_h, sizeof(unsigned long long) * ns,
                             cudaMemcpyHostToDevice, sim->st));
  }
  return IPC_OK;
}

void ccd(ipcsim* sim, const double* xv, const double* pv) {
  if (sim->P.broad_phase == IPC_BROAD_ALL_PAIRS)
    launch_ccd_brute(sim->st, sim->S, xv, pv, sim->P.s_ccd, ACCD_MAX_ITER, &sim->sc_dev->alpha, &sim->sc_dev->n_ccd);
  else
    launch_ccd_bvh(sim->st, sim->S, xv, pv, sim->P.s_ccd, ACCD_MAX_ITER, sim->tri_tree, sim->edge_tree,
                   &sim->sc_dev->alpha, &sim->sc_dev->n_ccd, &sim->sc_dev->flags);
}

// Sort the leaves and rebuild both hierarchies at xv (once per step; iterates refit).
void rebuild_trees(ipcsim* sim, const double* xv) {
  if (sim->P.broad_phase != IPC_BROAD_ALL_PAIRS) bvh_rebuild(sim->st, sim->S, xv, sim->bvh_pad, sim->tri_tree, sim->edge_tree);
}

ipc_status sync_scalars(ipcsim* sim) {
  CUDA_TRY(cudaMemcpyAsync(sim->sc_host, sim->sc_dev, sizeof(ipcsim::Scal), cudaMemcpyDeviceToHost, sim->st));
  if (sim->n_scenes > 1) {
    const int ns = sim->n_scenes;
    CUDA_TRY(cudaMemcpyAsync(sim->E_sc_h, sim->E_sc_dev, sizeof(acc_t) * 24 * ns, cudaMemcpyDeviceToHost, sim->st));
    CUDA_TRY(cudaMemcpyAsync(sim->alpha_sc_h, sim->alpha_sc_dev, sizeof(unsigned long long) * ns,
                             cudaMemcpyDeviceToHost, sim->st));
    CUDA_TRY(cudaMemcpyAsync(sim->pn_sc_h, sim->pn_sc_dev, sizeof(unsigned long long) * 2 * ns,
                             cudaMemcpyDeviceToHost, sim->st));
    CUDA_TRY(cudaMemcpyAsync(sim->min_sc_h.data(), sim->min_sc_dev, sizeof(unsigned long long) * ns,
                             cudaMemcpyDeviceToHost, sim->st));
  }
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  for (int k = 0; k < 8; ++k) sim->E_h[k] = acc_value(sim->sc_host->E + 3 * k);
  if (sim->n_scenes > 1) {
    sim->E_sc_v.resize(8 * (size_t)sim->n_scenes);
    for (size_t k = 0; k < sim->E_sc_v.size(); ++k) sim->E_sc_v[k] = acc_value(sim->E_sc_h + 3 * k);
  }
  prof_collect(sim);
  return IPC_OK;
}

// E: inertia, elastic, barrier, friction, stitch, ABD orthogonality, joints
double total_energy(const ipcsim* sim, const double* E) {
  double dt2 = sim->P.dt * sim->P.dt;
  return E[0] + dt2 * (E[1] + E[2] + E[3] + E[4] + E[5] + E[6]);
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof(d));
  return d;
}
unsigned long long double_bits(double d) {
  unsigned long long b;
  std::memcpy(&b, &d, sizeof(b));
  return b;
}

// Energy of the incremental potential at (zq, xkq) with positions xvq (computed here).
ipc_status energy_at(ipcsim* sim, const double* zq, const double* xkq, double* xvq, double* E_out, int* n_pairs) {
  const DevScene& S = sim->S;
  double dt2 = sim->P.dt * sim->P.dt;
  launch_vertex_positions(sim->st, S, zq, xkq, xvq);
  for (;;) {
    CUDA_TRY(cudaMemsetAsync(sim->sc_dev->E, 0, sizeof(sim->sc_dev->E), sim->st));
    if (sim->n_scenes > 1) CUDA_TRY(cudaMemsetAsync(sim->E_sc_dev, 0, sizeof(acc_t) * 24 * sim->n_scenes, sim->st));
    unsigned long long big = double_bits(1e300);
    CUDA_TRY(cudaMemcpyAsync(&sim->sc_dev->min_s, &big, sizeof(big), cudaMemcpyHostToDevice, sim->st));
    active_set(sim, xvq);
    launch_inertia(sim->st, S, zq, sim->z_tilde, nullptr, sim->sc_dev->E + 0, 0);
    launch_elastic(sim->st, S, xvq, dt2, 0, 0, nullptr, nullptr, sim->sc_dev->E + 3);
    launch_barrier(sim->st, pair_grid(sim->cap), S, xvq, sim->rec, &sim->sc_dev->n_pairs, sim->cap, sim->sh,
                   sim->kappa, dt2, 0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, sim->sc_dev->E + 6,
                   &sim->sc_dev->min_s);
    if (sim->P.mu > 0)
      launch_friction(sim->st, S, xvq, sim->xv_t, sim->n_fric, sim->f_ids, sim->f_w, sim->f_n, sim->f_lam, sim->P.mu,
                      sim->P.eps_v * sim->P.dt, dt2, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                      sim->sc_dev->E + 9);
    launch_stitch(sim->st, S, xvq, sim->stitch_hat, sim->k_c, dt2, 0, nullptr, sim->sc_dev->E + 12);
    launch_abd_orth(sim->st, S, zq, sim->P.kappa_A, dt2, 0, 0, nullptr, nullptr, sim->sc_dev->E + 15);
    launch_joints(sim->st, S, zq, dt2, 0, nullptr, nullptr, sim->sc_dev->E + 18);
    ipc_status s = sync_scalars(sim);
    if (s) return s;
    if (sim->sc_host->flags & ERRF_BVH) { sim->err = "BVH traversal stack overflow"; return IPC_ERR_BVH_OVERFLOW; }
    if (sim->sc_host->flags & ERRF_ACC) { sim->err = "an energy term is not finite or exceeds 2^94"; return IPC_ERR_NAN; }
    if (sim->sc_host->n_pairs > sim->cap) {
      if ((s = grow_pairs(sim, sim->sc_host->n_pairs))) return s;
      continue;
    }
    break;
  }
  *E_out = total_energy(sim, sim->E_h);
  if (n_pairs) *n_pairs = sim->sc_host->n_pairs;
  return IPC_OK;
}

}  // namespace

// Read access for the other translation units of this library.
ipc_status sim_internal_scene(ipcsim* sim, const ipc::DevScene** S, void** stream, double* sh, double* kappa,
                              std::string** err) {
  if (!sim) return IPC_ERR_ARG;
  *S = &sim->S;
  *stream = (void*)sim->st;
  *sh = sim->sh;
  *kappa = sim->kappa;
  *err = &sim->err;
  return IPC_OK;
}

extern "C" {

unsigned long long sim_kernel_launches(void) { return __atomic_load_n(&g_kernel_launches, __ATOMIC_RELAXED); }

const char* sim_last_error(const ipcsim* sim) { return sim ? sim->err.c_str() : g_create_error.c_str(); }

void sim_destroy(ipcsim* sim) {
  if (!sim) return;
  if (sim->st) cudaStreamSynchronize(sim->st);
  for (auto& a : sim->allocs) sim->mem.put(a.first, a.second);
  sim->allocs.clear();
  bvh_free(sim->tri_tree, sim->mem);
  bvh_free(sim->edge_tree, sim->mem);
  for (auto& e : sim->ev)
    if (e) cudaEventDestroy(e);
  if (sim->sc_host) cudaFreeHost(sim->sc_host);
  if (sim->E_sc_h) cudaFreeHost(sim->E_sc_h);
  if (sim->pcg_skip_h) cudaFreeHost(sim->pcg_skip_h);
  delete sim;
}

// Build a simulator for the scene D.  For a batch, D is the concatenation of
// n_scenes independent scenes and tet_scene / abd_scene / kin_scene give the
// scene of every tet, ABD body and kinematic body (NULL: all scene 0).
static ipc_status create_impl(const ipc_scene_desc* D, const ipc_params* params, const ipc_allocator* A, void* stream,
                              ipcsim** out, int n_scenes, const int* tet_scene, const int* abd_scene,
                              const int* kin_scene) {
  if (!out) return IPC_ERR_ARG;
  *out = nullptr;
  if (!D || !params) return IPC_ERR_ARG;
  if (A && (!A->alloc || !A->free)) {
    g_create_error = "allocator needs both alloc and free";
    return IPC_ERR_ARG;
  }
  ipcsim* sim = new ipcsim();
  sim->P = *params;
  sim->st = (cudaStream_t)stream;
  sim->mem.st = sim->st;
  if (A) {
    sim->mem.alloc_fn = A->alloc;
    sim->mem.free_fn = A->free;
    sim->mem.ctx = A->ctx;
  }
  auto fail = [&](ipc_status s, const std::string& msg) {
    if (!msg.empty()) sim->err = msg;
    g_create_error = sim->err;
    sim_destroy(sim);
    return s;
  };
  const ipc_params& P = sim->P;
  if (!(P.dt > 0) || !(P.dhat > 0) || D->n_fem_verts < 0 || D->n_tets < 0 || D->n_abd < 0 || D->n_kin < 0 ||
      D->n_stitch < 0)
    return fail(IPC_ERR_ARG, "invalid parameters or sizes");
  if ((D->n_tets > 0 && (!D->tets_host || !D->fem_X_host || !D->logE_host || !D->nu_host || !D->rho_host)))
    return fail(IPC_ERR_ARG, "missing FEM arrays");
  const int nj = D->n_joints;
  if (nj < 0 || (nj > 0 && (!D->joint_body_host || !D->joint_kind_host || !D->joint_vec_host || !D->joint_k_host ||
                            !D->joint_t_host)))
    return fail(IPC_ERR_ARG, "invalid joint arrays");
  for (int j = 0; j < nj; ++j) {
    const int a = D->joint_body_host[2 * j], b = D->joint_body_host[2 * j + 1];
    bool ok = a >= 0 && a < D->n_abd && b >= -1 && b < D->n_abd && std::isfinite(D->joint_k_host[j]) &&
              D->joint_k_host[j] >= 0;
    for (int s = 0; s < 2; ++s) ok = ok && (D->joint_kind_host[2 * j + s] == 0 || D->joint_kind_host[2 * j + s] == 1);
    for (int c = 0; c < 6; ++c) ok = ok && std::isfinite(D->joint_vec_host[6 * j + c]);
    for (int c = 0; c < 3; ++c) ok = ok && std::isfinite(D->joint_t_host[3 * j + c]);
    if (!ok) return fail(IPC_ERR_ARG, "joint " + std::to_string(j) + ": body, kind or value out of range");
  }

  const int nf = D->n_fem_verts, nt = D->n_tets, nab = D->n_abd, nkb = D->n_kin;
  sim->nf = nf; sim->nt = nt; sim->nab = nab; sim->nkb = nkb;
  for (int d = 0; d < 3; ++d) sim->grav[d] = D->gravity[d];

  // ---------------- FEM preparation
  if (n_scenes < 1) return fail(IPC_ERR_ARG, "n_scenes must be positive");
  std::vector<double> B(9 * (size_t)nt), vol(nt), mu(nt), lam(nt), mass(nf, 0.0);
  double Emax = 0.0;
  std::vector<double> Emax_s(n_scenes, 0.0);
  for (int e = 0; e < nt; ++e) {
    const int* t = D->tets_host + 4 * e;
    for (int a = 0; a < 4; ++a)
      if (t[a] < 0 || t[a] >= nf) return fail(IPC_ERR_ARG, "tet vertex id out of range");
    const double* X0 = D->fem_X_host + 3 * t[0];
    double Dm[9];
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i) Dm[3 * i + k] = D->fem_X_host[3 * t[k + 1] + i] - X0[i];
    double det;
    inv3(Dm, &B[9 * e], det);
    if (!(det > 0)) return fail(IPC_ERR_INVERTED, "rest tetrahedron " + std::to_string(e) + " is inverted or degenerate");
    vol[e] = det / 6.0;
    double E = std::exp(D->logE_host[e]), nu = D->nu_host[e];
    mu[e] = E / (2 * (1 + nu));
    // model parameter: first Lame parameter + mu (small-strain limit = linear material with E, nu)
    lam[e] = E * nu / ((1 + nu) * (1 - 2 * nu)) + mu[e];
    Emax = std::max(Emax, E);
    int sc_e = tet_scene ? tet_scene[e] : 0;
    Emax_s[sc_e] = std::max(Emax_s[sc_e], E);
    for (int a = 0; a < 4; ++a) mass[t[a]] += D->rho_host[e] * vol[e] / 4.0;
  }
  // surface faces: tet faces used once, outward (same face enumeration order for every run)
  std::vector<int> fem_surf;
  {
    const int fo[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
    std::unordered_map<unsigned long long, int> cnt;
    cnt.reserve(4 * (size_t)nt);
    auto key = [](int a, int b, int c) {
      int v[3] = {a, b, c};
      std::sort(v, v + 3);
      return ((unsigned long long)v[0] << 42) | ((unsigned long long)v[1] << 21) | (unsigned long long)v[2];
    };
    for (int f = 0; f < 4; ++f)
      for (int e = 0; e < nt; ++e) {
        const int* t = D->tets_host + 4 * e;
        cnt[key(t[fo[f][0]], t[fo[f][1]], t[fo[f][2]])]++;
      }
    for (int f = 0; f < 4; ++f)
      for (int e = 0; e < nt; ++e) {
        const int* t = D->tets_host + 4 * e;
        int a = t[fo[f][0]], b = t[fo[f][1]], c = t[fo[f][2]];
        if (cnt[key(a, b, c)] == 1) { fem_surf.push_back(a); fem_surf.push_back(b); fem_surf.push_back(c); }
      }
  }

  // ---------------- bodies and vertices
  std::vector<int> fem_vbody(nf, 0);
  int n_fem_bodies = 0;
  for (int e = 0; e < nt; ++e) {
    int b = D->fem_body_host ? D->fem_body_host[e] : 0;
    n_fem_bodies = std::max(n_fem_bodies, b + 1);
    for (int a = 0; a < 4; ++a) fem_vbody[D->tets_host[4 * e + a]] = b;
  }
  if (nt == 0 && nf > 0) n_fem_bodies = 1;
  std::vector<int> body_scene(n_fem_bodies, 0);
  for (int e = 0; e < nt; ++e)
    body_scene[D->fem_body_host ? D->fem_body_host[e] : 0] = tet_scene ? tet_scene[e] : 0;
  int na_v = 0, nk = 0;
  for (int i = 0; i < nab; ++i) na_v += D->abd_nverts_host[i];
  for (int i = 0; i < nkb; ++i) nk += D->kin_nverts_host[i];
  const int nv = nf + na_v + nk;
  sim->na_v = na_v; sim->nk = nk; sim->nv = nv;
  const int n_nodes = nf + 4 * nab;
  sim->n_nodes = n_nodes;
  std::vector<int> vkind(nv), vbody(nv), vabd(nv, -1), bkind;
  std::vector<double> xbar(3 * (size_t)nv);
  for (int b = 0; b < n_fem_bodies; ++b) bkind.push_back(VK_FEM);
  for (int v = 0; v < nf; ++v) {
    vkind[v] = VK_FEM; vbody[v] = fem_vbody[v];
    for (int d = 0; d < 3; ++d) xbar[3 * v + d] = D->fem_X_host[3 * v + d];
  }
  std::vector<int> tris_all;
  tris_all.insert(tris_all.end(), fem_surf.begin(), fem_surf.end());
  std::vector<double> abd_S(16 * (size_t)nab), abd_vol(nab);
  {
    int off = nf, xo = 0, to = 0;
    for (int i = 0; i < nab; ++i) {
      int nvb = D->abd_nverts_host[i], ntb = D->abd_ntris_host[i];
      int bid = (int)bkind.size();
      bkind.push_back(VK_ABD);
      body_scene.push_back(abd_scene ? abd_scene[i] : 0);
      const double* X = D->abd_X_host + 3 * xo;
      const int* T = D->abd_tris_host + 3 * to;
      // volume moments of the closed outward mesh: signed tets (origin, a, b, c)
      double V = 0, f1[3] = {0, 0, 0}, f2[9] = {0};
      for (int t = 0; t < ntb; ++t) {
        const double *a = X + 3 * T[3 * t], *b = X + 3 * T[3 * t + 1], *c = X + 3 * T[3 * t + 2];
        double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
        double Vt = (a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]) / 6.0;
        V += Vt;
        double s[3];
        for (int d = 0; d < 3; ++d) {
          s[d] = a[d] + b[d] + c[d];
          f1[d] += Vt * s[d] / 4.0;
        }
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) f2[3 * p + q] += Vt / 20.0 * (a[p] * a[q] + b[p] * b[q] + c[p] * c[q] + s[p] * s[q]);
      }
      if (!(V > 0)) return fail(IPC_ERR_ARG, "ABD mesh must be closed and outward oriented");
      double rho = D->abd_rho_host[i];
      double* Sb = &abd_S[16 * i];
      Sb[0] = rho * V;
      for (int d = 0; d < 3; ++d) { Sb[1 + d] = rho * f1[d]; Sb[4 * (1 + d)] = rho * f1[d]; }
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) Sb[4 * (1 + p) + 1 + q] = rho * f2[3 * p + q];
      abd_vol[i] = V;
      for (int v = 0; v < nvb; ++v) {
        int gv = off + v;
        vkind[gv] = VK_ABD; vbody[gv] = bid; vabd[gv] = i;
        for (int d = 0; d < 3; ++d) xbar[3 * gv + d] = X[3 * v + d];
      }
      for (int t = 0; t < 3 * ntb; ++t) tris_all.push_back(off + T[t]);
      off += nvb; xo += nvb; to += ntb;
    }
  }
  std::vector<int> kin_vbody(nk);
  {
    int off = nf + na_v, xo = 0, to = 0;
    for (int i = 0; i < nkb; ++i) {
      int nvb = D->kin_nverts_host[i], ntb = D->kin_ntris_host[i];
      int bid = (int)bkind.size();
      bkind.push_back(VK_KIN);
      body_scene.push_back(kin_scene ? kin_scene[i] : 0);
      for (int v = 0; v < nvb; ++v) {
        int gv = off + v;
        vkind[gv] = VK_KIN; vbody[gv] = bid;
        kin_vbody[gv - nf - na_v] = i;
        for (int d = 0; d < 3; ++d) xbar[3 * gv + d] = D->kin_X_host[3 * (xo + v) + d];
      }
      for (int t = 0; t < 3 * ntb; ++t) tris_all.push_back(off + D->kin_tris_host[3 * to + t]);
      off += nvb; xo += nvb; to += ntb;
    }
  }
  sim->nbody = (int)bkind.size();
  // edges: unique sorted vertex pairs in lexicographic order; surface vertices sorted unique
  std::vector<std::pair<int, int>> ev;
  ev.reserve(tris_all.size());
  for (size_t t = 0; t + 2 < tris_all.size(); t += 3)
    for (int k = 0; k < 3; ++k) {
      int a = tris_all[t + k], b = tris_all[t + (k + 1) % 3];
      ev.push_back({std::min(a, b), std::max(a, b)});
    }
  std::sort(ev.begin(), ev.end());
  ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
  std::vector<int> edges;
  for (auto& e : ev) { edges.push_back(e.first); edges.push_back(e.second); }
  std::vector<int> sv(tris_all.begin(), tris_all.end());
  std::sort(sv.begin(), sv.end());
  sv.erase(std::unique(sv.begin(), sv.end()), sv.end());
  std::vector<double> edge_rest_sq(ev.size());
  std::vector<double> ell_sum(n_scenes, 0.0), vol_ell(n_scenes, 0.0);
  std::vector<int> ell_n(n_scenes, 0), vol_n(n_scenes, 0);
  for (size_t k = 0; k < ev.size(); ++k) {
    double s = 0;
    for (int d = 0; d < 3; ++d) {
      double q = xbar[3 * ev[k].first + d] - xbar[3 * ev[k].second + d];
      s += q * q;
    }
    edge_rest_sq[k] = s;
    if (ev[k].first < nf && ev[k].second < nf) {
      int sc_k = body_scene[vbody[ev[k].first]];
      ell_sum[sc_k] += std::sqrt(s);
      ++ell_n[sc_k];
    }
  }
  for (int e = 0; e < nt; ++e) {
    int sc_e = tet_scene ? tet_scene[e] : 0;
    vol_ell[sc_e] += std::cbrt(vol[e]);
    ++vol_n[sc_e];
  }
  // per-scene barrier stiffness kbar / B''(dhat / 2), kbar = E_max * mean soft surface edge, and stitch stiffness
  std::vector<double> scene_kappa(n_scenes), scene_kc(n_scenes);
  for (int sc_i = 0; sc_i < n_scenes; ++sc_i) {
    double ell = ell_n[sc_i] ? ell_sum[sc_i] / ell_n[sc_i] : (vol_n[sc_i] ? vol_ell[sc_i] / vol_n[sc_i] : P.dhat);
    double Em = Emax_s[sc_i] > 0 ? Emax_s[sc_i] : 1e5;
    scene_kappa[sc_i] = P.kappa > 0 ? P.kappa : Em * ell / barrier_dd(0.5 * P.dhat, P.dhat);
    scene_kc[sc_i] = P.k_c > 0 ? P.k_c : 100.0 * Em * ell;
  }
  sim->h_sv = sv; sim->h_tris = tris_all; sim->h_edges = edges;
  sim->sh = P.dhat * P.dhat;
  sim->kappa = scene_kappa[0];
  sim->k_c = scene_kc[0];
  {
    const double fmax = P.kappa_max_factor > 0 ? P.kappa_max_factor : 100.0;
    sim->kappa_cur = scene_kappa;
    sim->kappa_max.resize(n_scenes);
    for (int k = 0; k < n_scenes; ++k) sim->kappa_max[k] = fmax * scene_kappa[k];
    sim->s_prev.assign(n_scenes, INFINITY);
  }
  sim->n_scenes = n_scenes;
  // L_bbox over the free bodies at the initial state, per scene; the Newton test uses the smallest
  {
    std::vector<double> lo(3 * n_scenes, 1e300), hi(3 * n_scenes, -1e300);
    for (int v = 0; v < nf; ++v) {
      int sc_v = body_scene[vbody[v]];
      for (int d = 0; d < 3; ++d) {
        lo[3 * sc_v + d] = std::min(lo[3 * sc_v + d], D->fem_X_host[3 * v + d]);
        hi[3 * sc_v + d] = std::max(hi[3 * sc_v + d], D->fem_X_host[3 * v + d]);
      }
    }
    int off = nf;
    for (int i = 0; i < nab; ++i) {
      const double* q = D->abd_q0_host + 12 * i;
      int sc_v = abd_scene ? abd_scene[i] : 0;
      for (int v = 0; v < D->abd_nverts_host[i]; ++v) {
        const double* xb = &xbar[3 * (off + v)];
        for (int d = 0; d < 3; ++d) {
          double x = q[d] + q[3 + d] * xb[0] + q[6 + d] * xb[1] + q[9 + d] * xb[2];
          lo[3 * sc_v + d] = std::min(lo[3 * sc_v + d], x);
          hi[3 * sc_v + d] = std::max(hi[3 * sc_v + d], x);
        }
      }
      off += D->abd_nverts_host[i];
    }
    sim->L = 0;
    for (int sc_i = 0; sc_i < n_scenes; ++sc_i) {
      if (lo[3 * sc_i] > hi[3 * sc_i]) continue;
      double s2 = 0;
      for (int d = 0; d < 3; ++d) s2 += (hi[3 * sc_i + d] - lo[3 * sc_i + d]) * (hi[3 * sc_i + d] - lo[3 * sc_i + d]);
      double Ls = std::sqrt(s2);
      sim->L = sim->L > 0 ? std::min(sim->L, Ls) : Ls;
    }
  }

  // ---------------- BSR pattern: diagonal, tet couplings, ABD 4x4 grids
  std::vector<std::vector<int>> rows(n_nodes);
  for (int i = 0; i < n_nodes; ++i) rows[i].push_back(i);
  for (int e = 0; e < nt; ++e) {
    const int* t = D->tets_host + 4 * e;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) rows[t[a]].push_back(t[b]);
  }
  for (int i = 0; i < nab; ++i)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) rows[nf + 4 * i + a].push_back(nf + 4 * i + b);
  // joints couple the pseudo-nodes of their two bodies
  for (int j = 0; j < nj; ++j) {
    const int ba = D->joint_body_host[2 * j], bb = D->joint_body_host[2 * j + 1];
    if (bb < 0 || bb == ba) continue;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        rows[nf + 4 * ba + a].push_back(nf + 4 * bb + b);
        rows[nf + 4 * bb + b].push_back(nf + 4 * ba + a);
      }
  }
  std::vector<int> row_ptr(n_nodes + 1, 0), col, diag(n_nodes);
  for (int i = 0; i < n_nodes; ++i) {
    auto& r = rows[i];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    row_ptr[i + 1] = row_ptr[i] + (int)r.size();
    for (int c : r) {
      if (c == i) diag[i] = (int)col.size();
      col.push_back(c);
    }
  }
  const int nnzb = (int)col.size();
  sim->nnzb = nnzb;
  auto find_blk = [&](int i, int j) {
    auto b = col.begin() + row_ptr[i], e = col.begin() + row_ptr[i + 1];
    return (int)(std::lower_bound(b, e, j) - col.begin());
  };
  std::vector<int> tet_blk(16 * (size_t)nt), abd_blk(16 * (size_t)nab);
  for (int e = 0; e < nt; ++e) {
    const int* t = D->tets_host + 4 * e;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) tet_blk[16 * e + 4 * a + b] = find_blk(t[a], t[b]);
  }
  for (int i = 0; i < nab; ++i)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) abd_blk[16 * i + 4 * a + b] = find_blk(nf + 4 * i + a, nf + 4 * i + b);
  // joint blocks: pseudo-node m of side s against pseudo-node n of side s'
  std::vector<int> jt_blk(64 * (size_t)nj, -1);
  for (int j = 0; j < nj; ++j)
    for (int p = 0; p < 8; ++p)
      for (int q = 0; q < 8; ++q) {
        const int bp = D->joint_body_host[2 * j + p / 4], bq = D->joint_body_host[2 * j + q / 4];
        if (bp >= 0 && bq >= 0) jt_blk[64 * j + 8 * p + q] = find_blk(nf + 4 * bp + p % 4, nf + 4 * bq + q % 4);
      }
  // elastic gathers: tets of every FEM block and of every FEM node, in tet order
  const int nfb = row_ptr[nf];
  sim->nfb = nfb;
  if (nt >= (1 << 27)) return fail(IPC_ERR_ARG, "too many tets (at most 2^27)");
  std::vector<int> eg_blk_ptr(nfb + 1, 0), eg_blk_ent(16 * (size_t)nt), eg_node_ptr(nf + 1, 0), eg_node_ent(4 * (size_t)nt);
  for (int e = 0; e < nt; ++e)
    for (int a = 0; a < 4; ++a) {
      ++eg_node_ptr[D->tets_host[4 * e + a] + 1];
      for (int b = 0; b < 4; ++b) ++eg_blk_ptr[tet_blk[16 * e + 4 * a + b] + 1];
    }
  for (int k = 0; k < nfb; ++k) eg_blk_ptr[k + 1] += eg_blk_ptr[k];
  for (int v = 0; v < nf; ++v) eg_node_ptr[v + 1] += eg_node_ptr[v];
  {
    std::vector<int> cb(eg_blk_ptr.begin(), eg_blk_ptr.end() - 1), cn(eg_node_ptr.begin(), eg_node_ptr.end() - 1);
    for (int e = 0; e < nt; ++e)
      for (int a = 0; a < 4; ++a) {
        eg_node_ent[cn[D->tets_host[4 * e + a]]++] = (e << 2) | a;
        for (int b = 0; b < 4; ++b) eg_blk_ent[cb[tet_blk[16 * e + 4 * a + b]]++] = (e << 4) | (a << 2) | b;
      }
  }
  // constant part: mass blocks and the stitch Hessian dt^2 k_c I
  std::vector<double> Hc(9 * (size_t)nnzb, 0.0);
  for (int v = 0; v < nf; ++v)
    for (int d = 0; d < 3; ++d) Hc[9 * (size_t)diag[v] + 4 * d] += mass[v];
  for (int i = 0; i < nab; ++i)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int d = 0; d < 3; ++d) Hc[9 * (size_t)abd_blk[16 * i + 4 * a + b] + 4 * d] += abd_S[16 * i + 4 * a + b];
  for (int k = 0; k < D->n_stitch; ++k) {
    int v = D->stitch_v_host[k];
    if (v < 0 || v >= nf || D->stitch_b_host[k] < 0 || D->stitch_b_host[k] >= nkb)
      return fail(IPC_ERR_ARG, "stitch index out of range");
    for (int d = 0; d < 3; ++d) Hc[9 * (size_t)diag[v] + 4 * d] += P.dt * P.dt * scene_kc[body_scene[vbody[v]]];
  }

  // ---------------- upload
  if (cudaStreamQuery(sim->st) == cudaErrorInvalidResourceHandle) return fail(IPC_ERR_ARG, "invalid stream");
  DevScene& S = sim->S;
  S.nf = nf; S.nt = nt; S.nab = nab; S.nkb = nkb; S.nv = nv; S.na_v = na_v; S.nk = nk; S.n_nodes = n_nodes;
  S.nsv = (int)sv.size(); S.ntri = (int)tris_all.size() / 3; S.nedge = (int)ev.size(); S.nbody = sim->nbody;
  {
    const int mx = std::max(std::max(nv, S.nsv), std::max(S.ntri, S.nedge));
    while (sim->prim_bits < 31 && (1LL << sim->prim_bits) <= mx) ++sim->prim_bits;
  }
  S.nnzb = nnzb;
  S.n_stitch = D->n_stitch;
  ipc_status s;
  {
    std::vector<int> tet_i(4 * (size_t)nt);
    for (size_t i = 0; i < tet_i.size(); ++i) tet_i[i] = D->tets_host[i];
    int* ptr;
    if ((s = upload(sim, &ptr, tet_i))) return fail(s, "");
    S.tets = (const int4*)ptr;
  }
  {
    double* dp; int* ip;
    if ((s = upload(sim, &dp, B))) return fail(s, ""); S.B = dp;
    if ((s = upload(sim, &dp, vol))) return fail(s, ""); S.vol = dp;
    if ((s = upload(sim, &dp, mu))) return fail(s, ""); S.mu = dp; sim->d_mu = dp;
    if ((s = upload(sim, &dp, lam))) return fail(s, ""); S.lam = dp; sim->d_lam = dp;
    sim->h_nu.assign(D->nu_host, D->nu_host + nt);
    sim->h_logE.assign(D->logE_host, D->logE_host + nt);
    if ((s = upload(sim, &ip, tet_blk))) return fail(s, ""); S.tet_blk = ip;
    S.nfb = nfb;
    if ((s = upload(sim, &ip, eg_blk_ptr))) return fail(s, ""); S.eg_blk_ptr = ip;
    if ((s = upload(sim, &ip, eg_blk_ent))) return fail(s, ""); S.eg_blk_ent = ip;
    if ((s = upload(sim, &ip, eg_node_ptr))) return fail(s, ""); S.eg_node_ptr = ip;
    if ((s = upload(sim, &ip, eg_node_ent))) return fail(s, ""); S.eg_node_ent = ip;
    if ((s = upload(sim, &ip, vkind))) return fail(s, ""); S.vkind = ip;
    if ((s = upload(sim, &ip, vbody))) return fail(s, ""); S.vbody = ip;
    if ((s = upload(sim, &ip, vabd))) return fail(s, ""); S.vabd = ip;
    if ((s = upload(sim, &dp, xbar))) return fail(s, ""); S.xbar = dp;
    if ((s = upload(sim, &ip, bkind))) return fail(s, ""); S.bkind = ip;
    if ((s = upload(sim, &ip, sv))) return fail(s, ""); S.sv = ip;
    if ((s = upload(sim, &ip, tris_all))) return fail(s, ""); S.tris = (const int3*)ip;
    if ((s = upload(sim, &ip, edges))) return fail(s, ""); S.edges = (const int2*)ip;
    if ((s = upload(sim, &dp, edge_rest_sq))) return fail(s, ""); S.edge_rest_sq = dp;
    if ((s = upload(sim, &dp, mass))) return fail(s, ""); S.node_mass = dp;
    if ((s = upload(sim, &dp, abd_S))) return fail(s, ""); S.abd_S = dp;
    if ((s = upload(sim, &dp, abd_vol))) return fail(s, ""); S.abd_vol = dp;
    if ((s = upload(sim, &ip, abd_blk))) return fail(s, ""); S.abd_blk = ip;
    if ((s = upload(sim, &ip, kin_vbody))) return fail(s, ""); S.kin_vbody = ip;
    std::vector<int> stv(D->stitch_v_host, D->stitch_v_host + D->n_stitch), stb(D->stitch_b_host, D->stitch_b_host + D->n_stitch);
    std::vector<double> stx(D->stitch_X_host, D->stitch_X_host + 3 * D->n_stitch);
    if ((s = upload(sim, &ip, stv))) return fail(s, ""); S.stitch_v = ip;
    if ((s = upload(sim, &ip, stb))) return fail(s, ""); S.stitch_b = ip;
    if ((s = upload(sim, &dp, stx))) return fail(s, ""); S.stitch_X = dp;
    S.nj = nj;
    sim->nj = nj;
    if (nj) {
      std::vector<int> jb(D->joint_body_host, D->joint_body_host + 2 * nj), jk(D->joint_kind_host, D->joint_kind_host + 2 * nj);
      std::vector<double> va(3 * (size_t)nj), vb(3 * (size_t)nj), jkk(D->joint_k_host, D->joint_k_host + nj),
          jt(D->joint_t_host, D->joint_t_host + 3 * nj);
      for (int j = 0; j < nj; ++j)
        for (int c = 0; c < 3; ++c) {
          va[3 * j + c] = D->joint_vec_host[6 * j + c];
          vb[3 * j + c] = D->joint_vec_host[6 * j + 3 + c];
        }
      if ((s = upload(sim, &ip, jb))) return fail(s, ""); S.jt_body = ip;
      if ((s = upload(sim, &ip, jk))) return fail(s, ""); S.jt_kind = ip;
      if ((s = upload(sim, &dp, va))) return fail(s, ""); S.jt_va = dp;
      if ((s = upload(sim, &sim->jt_vb, vb))) return fail(s, ""); S.jt_vb = sim->jt_vb;
      if ((s = upload(sim, &dp, jkk))) return fail(s, ""); S.jt_k = dp;
      if ((s = upload(sim, &sim->jt_t, jt))) return fail(s, ""); S.jt_t = sim->jt_t;
      if ((s = upload(sim, &ip, jt_blk))) return fail(s, ""); S.jt_blk = ip;
    }
    if ((s = upload(sim, &ip, row_ptr))) return fail(s, ""); S.bsr_row = ip;
    sim->h_row = row_ptr;
    if ((s = upload(sim, &ip, col))) return fail(s, ""); S.bsr_col = ip;
    if ((s = upload(sim, &ip, diag))) return fail(s, ""); S.bsr_diag = ip;
    if ((s = upload(sim, &sim->Hconst, Hc))) return fail(s, "");
    if ((s = upload(sim, &ip, body_scene))) return fail(s, ""); S.body_scene = ip;
    if ((s = upload(sim, &dp, scene_kappa))) return fail(s, ""); S.scene_kappa = dp; sim->d_scene_kappa = dp;
    if ((s = upload(sim, &dp, scene_kc))) return fail(s, ""); S.scene_kc = dp;
    S.n_scenes = n_scenes;
    if (n_scenes > 1) {
      // scene of every node: FEM vertices through their body, ABD pseudo-nodes through their body
      std::vector<int> node_scene(n_nodes);
      for (int i = 0; i < nf; ++i) node_scene[i] = body_scene[vbody[i]];
      for (int v = nf; v < nf + na_v; ++v)
        for (int t = 0; t < 4; ++t) node_scene[nf + 4 * vabd[v] + t] = body_scene[vbody[v]];
      if ((s = upload(sim, &ip, node_scene))) return fail(s, ""); S.node_scene = ip;
      sim->h_node_scene = node_scene;
      if ((s = dalloc(sim, &sim->d_pcg_skip, (size_t)n_scenes))) return fail(s, "");
      if ((s = dalloc(sim, &sim->d_pcg_sc_res, (size_t)n_scenes))) return fail(s, "");
      if (cudaMallocHost(&sim->pcg_skip_h, sizeof(int) * (size_t)n_scenes) != cudaSuccess)
        return fail(IPC_ERR_CUDA, "cudaMallocHost failed");
      if ((s = dalloc(sim, &sim->E_sc_dev, 24 * (size_t)n_scenes))) return fail(s, ""); S.E_sc = sim->E_sc_dev;
      if ((s = dalloc(sim, &sim->min_sc_dev, (size_t)n_scenes))) return fail(s, ""); S.min_sc = sim->min_sc_dev;
      sim->min_sc_h.assign(n_scenes, 0);
      if ((s = dalloc(sim, &sim->alpha_sc_dev, (size_t)n_scenes))) return fail(s, ""); S.alpha_sc = sim->alpha_sc_dev;
      if ((s = dalloc(sim, &sim->pn_sc_dev, 2 * (size_t)n_scenes))) return fail(s, ""); S.pn_sc = sim->pn_sc_dev;
      if ((s = dalloc(sim, &sim->alpha_trial_dev, (size_t)n_scenes))) return fail(s, "");
      S.alpha_trial = sim->alpha_trial_dev;
      void* hb = nullptr;
      if (cudaMallocHost(&hb, sizeof(acc_t) * 27 * (size_t)n_scenes) != cudaSuccess)
        return fail(IPC_ERR_CUDA, "cudaMallocHost failed");
      sim->E_sc_h = static_cast<acc_t*>(hb);
      sim->alpha_sc_h = sim->E_sc_h + 24 * (size_t)n_scenes;
      sim->pn_sc_h = sim->alpha_sc_h + n_scenes;
    }
  }
  // state
  const int ndof = 3 * n_nodes;
  {
    std::vector<double> z(ndof, 0.0), zd(ndof, 0.0);
    for (int i = 0; i < 3 * nf; ++i) {
      z[i] = D->fem_X_host[i];
      if (D->fem_V0_host) zd[i] = D->fem_V0_host[i];
    }
    for (int i = 0; i < nab; ++i)
      for (int k = 0; k < 12; ++k) z[3 * nf + 12 * i + k] = D->abd_q0_host[12 * i + k];
    if ((s = upload(sim, &sim->z, z))) return fail(s, "");
    if ((s = upload(sim, &sim->zd, zd))) return fail(s, "");
    sim->h_Tcur.assign(D->kin_T0_host, D->kin_T0_host + 12 * nkb);
    std::vector<double> xk(3 * (size_t)nk);
    for (int i = 0; i < nk; ++i) {
      const double* M = &sim->h_Tcur[12 * kin_vbody[i]];
      const double* xb = &xbar[3 * (nf + na_v + i)];
      for (int d = 0; d < 3; ++d) xk[3 * i + d] = M[4 * d] * xb[0] + M[4 * d + 1] * xb[1] + M[4 * d + 2] * xb[2] + M[4 * d + 3];
    }
    if ((s = upload(sim, &sim->xk, xk))) return fail(s, "");
  }
  double** bufs3n[] = {&sim->z_t, &sim->z_tilde, &sim->z_trial, &sim->g, &sim->gdir, &sim->rhs, &sim->p, &sim->y};
  for (auto b : bufs3n)
    if ((s = dalloc(sim, b, ndof))) return fail(s, "");
  double** bufsk[] = {&sim->xk_t, &sim->xk_hat, &sim->xk_trial, &sim->pD};
  for (auto b : bufsk)
    if ((s = dalloc(sim, b, 3 * (size_t)nk))) return fail(s, "");
  double** bufsv[] = {&sim->xv, &sim->xv_t, &sim->xv_trial, &sim->pv};
  for (auto b : bufsv)
    if ((s = dalloc(sim, b, 3 * (size_t)nv))) return fail(s, "");
  if ((s = dalloc(sim, &sim->stitch_hat, 3 * (size_t)D->n_stitch))) return fail(s, "");
  if ((s = dalloc(sim, &sim->Hval, 9 * (size_t)nnzb))) return fail(s, "");
  if ((s = dalloc(sim, &sim->Dc, 9 * (size_t)n_nodes))) return fail(s, "");
  if ((s = dalloc(sim, &sim->H_acc, 27 * (size_t)nnzb))) return fail(s, "");
  if ((s = dalloc(sim, &sim->el_tU, 78 * (size_t)nt))) return fail(s, "");
  if ((s = dalloc(sim, &sim->el_tG, 12 * (size_t)nt))) return fail(s, "");
  if ((s = dalloc(sim, &sim->Dc_acc, 27 * (size_t)n_nodes))) return fail(s, "");
  if ((s = dalloc(sim, &sim->g_acc, 3 * (size_t)ndof))) return fail(s, "");
  if ((s = dalloc(sim, &sim->gdir_acc, 3 * (size_t)ndof))) return fail(s, "");
  if ((s = dalloc(sim, &sim->gz_acc, 3 * (size_t)ndof))) return fail(s, "");
  if ((s = dalloc(sim, &sim->Dinv, 9 * (size_t)n_nodes))) return fail(s, "");
  if ((s = dalloc(sim, &sim->T_dev, 12 * (size_t)std::max(nkb, 1)))) return fail(s, "");
  if (P.precision != IPC_PREC_FP64 && P.precision != IPC_PREC_MIXED) return fail(IPC_ERR_ARG, "unknown precision");
  sim->pcg_grid_max = 4 * device_sms();  // sizes the partial-sum buffer: up to four CTAs per SM
  if ((s = dalloc(sim, &sim->pcg_op, 9 * (size_t)nnzb))) return fail(s, "");
  if ((s = dalloc(sim, &sim->pcg_vec, 9 * (size_t)ndof))) return fail(s, "");
  if ((s = dalloc(sim, &sim->inc_ptr, (size_t)nf + nab + 1))) return fail(s, "");
  if ((s = dalloc(sim, &sim->inc_cursor, (size_t)nf + nab + 1))) return fail(s, "");
  if ((s = dalloc(sim, &sim->inc_tiles, (size_t)(nf + nab + 1) / 4096 + 1))) return fail(s, "");
  if (nab) {
    if ((s = dalloc(sim, &sim->abd_ptr, (size_t)nab + 1))) return fail(s, "");
    if ((s = dalloc(sim, &sim->abd_cursor, (size_t)nab + 1))) return fail(s, "");
    if ((s = grow_abd_list(sim, std::max<long long>(4096, 12LL * (sim->cap + sim->fcap))))) return fail(s, "");
  }
  if (P.precision == IPC_PREC_MIXED)
    if ((s = dalloc(sim, &sim->Dinv32, 9 * (size_t)n_nodes))) return fail(s, "");
  if ((s = dalloc(sim, &sim->partial, pcg_partial_doubles(sim->pcg_grid_max)))) return fail(s, "");
  if ((s = dalloc(sim, &sim->sc_dev, 1))) return fail(s, "");
  S.err = &sim->sc_dev->flags;
  {
    acc_t* slots = nullptr;
    if ((s = dalloc(sim, &slots, 3 * (size_t)E_SLOTS))) return fail(s, "");
    S.e_slots = slots;
  }
  if (cudaMallocHost((void**)&sim->sc_host, sizeof(ipcsim::Scal)) != cudaSuccess) return fail(IPC_ERR_CUDA, "cudaMallocHost failed");
  std::memset(sim->sc_host, 0, sizeof(ipcsim::Scal));
  int cap0 = P.pair_capacity > 0 ? P.pair_capacity : std::max(1024, 2 * (S.nsv + S.nedge));
  const int pairs0 = (int)std::min<long long>(cap0 * 2 / 3 + 1, max_pairs(sim));
  if ((s = grow_pairs(sim, pairs0))) return fail(s, "");
  if ((s = grow_cand(sim, 4 * cap0))) return fail(s, "");
  if ((s = grow_fric(sim, pairs0))) return fail(s, "");
  if (cudaMemcpyAsync(sim->T_dev, sim->h_Tcur.data(), sizeof(double) * 12 * nkb, cudaMemcpyHostToDevice, sim->st) != cudaSuccess && nkb)
    return fail(IPC_ERR_CUDA, "upload of transforms failed");
  // broad phase: leaf boxes widened by slightly more than dhat, so that every
  // pair closer than dhat overlaps despite rounding of the widened bounds
  sim->bvh_pad = P.dhat * (1.0 + 1e-6);
  if (bvh_alloc(sim->tri_tree, S.ntri, sim->mem) != cudaSuccess || bvh_alloc(sim->edge_tree, S.nedge, sim->mem) != cudaSuccess)
    return fail(IPC_ERR_CUDA, "BVH allocation failed");
  // initial state must be intersection free: no pair at zero distance
  launch_vertex_positions(sim->st, S, sim->z, sim->xk, sim->xv);
  rebuild_trees(sim, sim->xv);
  cudaMemsetAsync(&sim->sc_dev->flags, 0, sizeof(int), sim->st);
  cull(sim, sim->xv);
  if (sync_scalars(sim)) return fail(IPC_ERR_CUDA, "");
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(IPC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(ce));
  if (sim->sc_host->n_pairs > sim->cap) {
    if ((s = grow_pairs(sim, sim->sc_host->n_pairs))) return fail(s, "");
    cull(sim, sim->xv);
    if (sync_scalars(sim)) return fail(IPC_ERR_CUDA, "");
  }
  {
    int n = std::min(sim->sc_host->n_pairs, sim->cap);
    std::vector<double> ss(n);
    if (n) cudaMemcpy(ss.data(), sim->rec_s, sizeof(double) * n, cudaMemcpyDeviceToHost);
    for (double v : ss)
      if (!(v > 0)) return fail(IPC_ERR_INTERSECTING, "initial state has a contact pair at zero distance");
  }
  *out = sim;
  return IPC_OK;
}

ipc_status sim_create(const ipc_scene_desc* D, const ipc_params* params, void* stream, ipcsim** out) {
  return create_impl(D, params, nullptr, stream, out, 1, nullptr, nullptr, nullptr);
}

static ipc_status batch_impl(const ipc_scene_desc* descs, int n, const ipc_params* params, const ipc_allocator* A,
                             void* stream, ipcsim** out);

ipc_status sim_create_batch(const ipc_scene_desc* descs, int n, const ipc_params* params, void* stream, ipcsim** out) {
  return batch_impl(descs, n, params, nullptr, stream, out);
}

ipc_status sim_create_with_allocator(const ipc_scene_desc* descs, int n, const ipc_params* params,
                                     const ipc_allocator* allocator, void* stream, ipcsim** out) {
  if (!allocator) return IPC_ERR_ARG;
  if (n == 1) return create_impl(descs, params, allocator, stream, out, 1, nullptr, nullptr, nullptr);
  return batch_impl(descs, n, params, allocator, stream, out);
}

ipc_status sim_memory(const ipcsim* sim, long long* out3) {
  if (!sim || !out3) return IPC_ERR_ARG;
  out3[0] = sim->mem.by_allocator;
  out3[1] = sim->mem.direct;
  out3[2] = sim->mem.bytes;
  return IPC_OK;
}

static ipc_status batch_impl(const ipc_scene_desc* descs, int n, const ipc_params* params, const ipc_allocator* A,
                             void* stream, ipcsim** out) {
  if (!out) return IPC_ERR_ARG;
  *out = nullptr;
  if (!descs || n <= 0 || !params) return IPC_ERR_ARG;
  std::vector<double> fX, fV0, logE, nu, rho, aX, arho, aq0, kX, kT0, stX, jvec, jk, jt;
  std::vector<int> tets, fbody, anv, antri, atris, knv, kntri, ktris, stv, stb, tet_scene, abd_scene, kin_scene, jbody,
      jkind;
  bool any_v0 = false;
  for (int k = 0; k < n; ++k) any_v0 |= descs[k].fem_V0_host != nullptr;
  int voff = 0, boff = 0, koff = 0;
  for (int k = 0; k < n; ++k) {
    const ipc_scene_desc& D = descs[k];
    if (D.n_fem_verts < 0 || D.n_tets < 0 || D.n_abd < 0 || D.n_kin < 0 || D.n_stitch < 0 || D.n_joints < 0)
      return IPC_ERR_ARG;
    if (D.n_joints > 0 && (!D.joint_body_host || !D.joint_kind_host || !D.joint_vec_host || !D.joint_k_host ||
                           !D.joint_t_host))
      return IPC_ERR_ARG;
    for (int j = 0; j < D.n_joints; ++j) {
      // bodies are shifted by the affine bodies of the scenes before; the world (-1) stays; ids out of the
      // scene's range are left out of range for create's check
      for (int s = 0; s < 2; ++s) {
        const int b = D.joint_body_host[2 * j + s];
        jbody.push_back(b >= 0 && b < D.n_abd ? b + (int)abd_scene.size() : (b == -1 ? -1 : -2));
        jkind.push_back(D.joint_kind_host[2 * j + s]);
      }
      jk.push_back(D.joint_k_host[j]);
    }
    if (D.n_joints) {
      jvec.insert(jvec.end(), D.joint_vec_host, D.joint_vec_host + 6 * D.n_joints);
      jt.insert(jt.end(), D.joint_t_host, D.joint_t_host + 3 * D.n_joints);
    }
    fX.insert(fX.end(), D.fem_X_host, D.fem_X_host + 3 * D.n_fem_verts);
    if (any_v0) {
      if (D.fem_V0_host) fV0.insert(fV0.end(), D.fem_V0_host, D.fem_V0_host + 3 * D.n_fem_verts);
      else fV0.insert(fV0.end(), 3 * (size_t)D.n_fem_verts, 0.0);
    }
    int nb = 0;
    for (int e = 0; e < D.n_tets; ++e) {
      for (int a = 0; a < 4; ++a) tets.push_back(D.tets_host[4 * e + a] + voff);
      int b = D.fem_body_host ? D.fem_body_host[e] : 0;
      fbody.push_back(b + boff);
      nb = std::max(nb, b + 1);
      tet_scene.push_back(k);
    }
    logE.insert(logE.end(), D.logE_host, D.logE_host + D.n_tets);
    nu.insert(nu.end(), D.nu_host, D.nu_host + D.n_tets);
    rho.insert(rho.end(), D.rho_host, D.rho_host + D.n_tets);
    int av = 0, at = 0;
    for (int i = 0; i < D.n_abd; ++i) {
      anv.push_back(D.abd_nverts_host[i]);
      antri.push_back(D.abd_ntris_host[i]);
      av += D.abd_nverts_host[i];
      at += D.abd_ntris_host[i];
      abd_scene.push_back(k);
    }
    if (D.n_abd) {
      aX.insert(aX.end(), D.abd_X_host, D.abd_X_host + 3 * av);
      atris.insert(atris.end(), D.abd_tris_host, D.abd_tris_host + 3 * at);
      arho.insert(arho.end(), D.abd_rho_host, D.abd_rho_host + D.n_abd);
      aq0.insert(aq0.end(), D.abd_q0_host, D.abd_q0_host + 12 * D.n_abd);
    }
    int kv = 0, kt = 0;
    for (int i = 0; i < D.n_kin; ++i) {
      knv.push_back(D.kin_nverts_host[i]);
      kntri.push_back(D.kin_ntris_host[i]);
      kv += D.kin_nverts_host[i];
      kt += D.kin_ntris_host[i];
      kin_scene.push_back(k);
    }
    if (D.n_kin) {
      kX.insert(kX.end(), D.kin_X_host, D.kin_X_host + 3 * kv);
      ktris.insert(ktris.end(), D.kin_tris_host, D.kin_tris_host + 3 * kt);
      kT0.insert(kT0.end(), D.kin_T0_host, D.kin_T0_host + 12 * D.n_kin);
    }
    for (int i = 0; i < D.n_stitch; ++i) {
      stv.push_back(D.stitch_v_host[i] + voff);
      stb.push_back(D.stitch_b_host[i] + koff);
    }
    if (D.n_stitch) stX.insert(stX.end(), D.stitch_X_host, D.stitch_X_host + 3 * D.n_stitch);
    voff += D.n_fem_verts;
    boff += (D.n_tets || D.n_fem_verts) ? std::max(nb, 1) : 0;
    koff += D.n_kin;
  }
  ipc_scene_desc M{};
  M.n_fem_verts = voff;
  M.fem_X_host = fX.data();
  M.fem_V0_host = any_v0 ? fV0.data() : nullptr;
  M.n_tets = (int)tet_scene.size();
  M.tets_host = tets.data();
  M.logE_host = logE.data();
  M.nu_host = nu.data();
  M.rho_host = rho.data();
  M.fem_body_host = fbody.data();
  M.n_abd = (int)abd_scene.size();
  M.abd_nverts_host = anv.data();
  M.abd_X_host = aX.data();
  M.abd_ntris_host = antri.data();
  M.abd_tris_host = atris.data();
  M.abd_rho_host = arho.data();
  M.abd_q0_host = aq0.data();
  M.n_kin = (int)kin_scene.size();
  M.kin_nverts_host = knv.data();
  M.kin_X_host = kX.data();
  M.kin_ntris_host = kntri.data();
  M.kin_tris_host = ktris.data();
  M.kin_T0_host = kT0.data();
  M.n_stitch = (int)stv.size();
  M.stitch_v_host = stv.data();
  M.stitch_b_host = stb.data();
  M.stitch_X_host = stX.data();
  M.n_joints = (int)jk.size();
  M.joint_body_host = jbody.data();
  M.joint_kind_host = jkind.data();
  M.joint_vec_host = jvec.data();
  M.joint_k_host = jk.data();
  M.joint_t_host = jt.data();
  for (int d = 0; d < 3; ++d) M.gravity[d] = descs[0].gravity[d];
  return create_impl(&M, params, A, stream, out, n, tet_scene.data(), abd_scene.data(), kin_scene.data());
}

ipc_status sim_sizes(const ipcsim* sim, int* o) {
  if (!sim || !o) return IPC_ERR_ARG;
  o[0] = sim->nf; o[1] = sim->nt; o[2] = sim->nab; o[3] = sim->nkb;
  o[4] = (int)sim->h_tris.size() / 3; o[5] = (int)sim->h_edges.size() / 2; o[6] = (int)sim->h_sv.size();
  o[7] = sim->n_nodes; o[8] = sim->nnzb;
  return IPC_OK;
}

ipc_status sim_scalars(const ipcsim* sim, double* o) {
  if (!sim || !o) return IPC_ERR_ARG;
  o[0] = sim->kappa; o[1] = sim->k_c; o[2] = sim->L; o[3] = sim->P.dhat;
  return IPC_OK;
}

ipc_status sim_surface(const ipcsim* sim, int* sv, int* tris, int* edges) {
  if (!sim) return IPC_ERR_ARG;
  if (sv) std::memcpy(sv, sim->h_sv.data(), sizeof(int) * sim->h_sv.size());
  if (tris) std::memcpy(tris, sim->h_tris.data(), sizeof(int) * sim->h_tris.size());
  if (edges) std::memcpy(edges, sim->h_edges.data(), sizeof(int) * sim->h_edges.size());
  return IPC_OK;
}

}  // extern "C"

namespace {

// The body of sim_step.  Every return after the start of the step leaves the
// state to the caller (sim_step), which puts it back to x_t on any error:
// `started` is set once z_t and xk_t hold the state at the start of the step.
// Adaptive barrier stiffness after an accepted Newton iterate: s_it[k] is the smallest squared distance of
// scene k's iterate (its assembly), done[k] != 0 skips a scene.  kappa doubles, up to its cap, when s_it is
// below (kappa_dmin dhat)^2 and not larger than the previous iterate's.
ipc_status adapt_kappa(ipcsim* sim, const std::vector<double>& s_it, const std::vector<char>* done) {
  const ipc_params& P = sim->P;
  if (!P.kappa_adaptive) return IPC_OK;
  const double dmin = (P.kappa_dmin > 0 ? P.kappa_dmin : 1e-2) * P.dhat;
  bool changed = false;
  for (int k = 0; k < sim->n_scenes; ++k) {
    if (done && !done->empty() && (*done)[k]) continue;
    if (s_it[k] < dmin * dmin && s_it[k] <= sim->s_prev[k] && sim->kappa_cur[k] < sim->kappa_max[k]) {
      sim->kappa_cur[k] = std::min(2.0 * sim->kappa_cur[k], sim->kappa_max[k]);
      changed = true;
    }
    sim->s_prev[k] = s_it[k];
  }
  if (changed) {
    sim->kappa = sim->kappa_cur[0];
    CUDA_TRY(cudaMemcpyAsync(sim->d_scene_kappa, sim->kappa_cur.data(), sizeof(double) * sim->n_scenes,
                             cudaMemcpyHostToDevice, sim->st));
    CUDA_TRY(cudaStreamSynchronize(sim->st));
  }
  return IPC_OK;
}

ipc_status step_body(ipcsim* sim, const double* kin_T_next, ipc_step_stats& st, bool& started) {
  const DevScene& S = sim->S;
  const ipc_params& P = sim->P;
  const int ndof = 3 * sim->n_nodes, nk3 = 3 * sim->nk;
  const double dt = P.dt, dt2 = dt * dt;
  cudaStream_t cs = sim->st;
  if (sim->nkb) CUDA_TRY(cudaMemcpyAsync(sim->T_dev, kin_T_next, sizeof(double) * 12 * sim->nkb, cudaMemcpyHostToDevice, cs));
  sim->kappa_step = sim->kappa_cur;
  sim->s_prev.assign(sim->n_scenes, INFINITY);
  launch_predict(cs, S, sim->z, sim->zd, dt, sim->grav, sim->z_t, sim->z_tilde);
  if (nk3) CUDA_TRY(cudaMemcpyAsync(sim->xk_t, sim->xk, sizeof(double) * nk3, cudaMemcpyDeviceToDevice, cs));
  started = true;
  launch_kin_targets(cs, S, sim->T_dev, sim->xk_hat, sim->stitch_hat);
  launch_vertex_positions(cs, S, sim->z, sim->xk, sim->xv);
  CUDA_TRY(cudaMemcpyAsync(sim->xv_t, sim->xv, sizeof(double) * 3 * sim->nv, cudaMemcpyDeviceToDevice, cs));
  rebuild_trees(sim, sim->xv);
  CUDA_TRY(cudaMemsetAsync(sim->sc_dev, 0, sizeof(ipcsim::Scal), cs));
  ipc_status s = IPC_OK;
  sim->cand_valid = false;
  sim->co_built_this_step = false;
  sim->co_step_iters = sim->co_step_solves = 0;
  bool rec_current = false;  // sim->rec holds the active set at the current iterate
  const bool sweep = P.broad_phase != IPC_BROAD_ALL_PAIRS;
  // friction lag on the pairs active at x_t
  sim->n_fric = 0;
  if (P.mu > 0) {
    for (;;) {
      cull(sim, sim->xv);
      if ((s = sync_scalars(sim))) return s;
      if (sim->sc_host->n_pairs > sim->cap) { if ((s = grow_pairs(sim, sim->sc_host->n_pairs))) return s; continue; }
      break;
    }
    int n = sim->sc_host->n_pairs;
    if (n > sim->fcap && (s = grow_fric(sim, n))) return s;
    launch_friction_lag(cs, pair_grid(sim->cap), S, sim->xv, sim->rec, &sim->sc_dev->n_pairs, sim->cap, sim->sh,
                        sim->kappa, sim->f_ids, sim->f_w, sim->f_n, sim->f_lam);
    sim->n_fric = n;
    rec_current = true;
  }
  st.n_friction_pairs = sim->n_fric;
  const double tol_abs = P.newton_tol * dt * sim->L;
  const int max_pcg = P.max_pcg > 0 ? P.max_pcg : (int)(10.0 * std::sqrt((double)ndof)) + 100;
  bool converged = false;
  int it = 0;
  std::vector<char> scene_done;  // batches: scenes whose Newton iteration has converged
  auto finish = [&](ipc_status code, const char* msg) {
    sim->err = msg;
    return code;
  };
  while (it < P.max_newton) {
    // ---- assemble gradient, Hessian and Dirichlet coupling at the current iterate
    if ((s = reset_iteration_scalars(sim))) return s;
    if ((s = assembly_begin(sim))) return s;
    launch_vertex_positions(cs, S, sim->z, sim->xk, sim->xv);
    launch_sub(cs, nk3, sim->xk_hat, sim->xk, sim->pD);
    if (!rec_current) {
      prof_begin(sim, PROF_CULL);
      cull(sim, sim->xv);
      prof_end(sim, PROF_CULL);
    }
    launch_inertia(cs, S, sim->z, sim->z_tilde, sim->g_acc, sim->sc_dev->E + 0, 1);
    prof_begin(sim, PROF_ELASTIC);
    launch_elastic_assembly(cs, S, sim->xv, dt2, 1, sim->g_acc, sim->Hconst, sim->Hval, sim->sc_dev->E + 3,
                            P.precision == IPC_PREC_MIXED, sim->el_tU, sim->el_tG);
    prof_end(sim, PROF_ELASTIC);
    launch_stitch(cs, S, sim->xv, sim->stitch_hat, sim->k_c, dt2, 1, sim->g_acc, sim->sc_dev->E + 12);
    launch_abd_orth(cs, S, sim->z, P.kappa_A, dt2, 2, 1, sim->g_acc, sim->H_acc, sim->sc_dev->E + 15);
    launch_joints(cs, S, sim->z, dt2, 2, sim->g_acc, sim->H_acc, sim->sc_dev->E + 18);
    prof_begin(sim, PROF_BARRIER);
    launch_barrier(cs, pair_grid(sim->cap), S, sim->xv, sim->rec, &sim->sc_dev->n_pairs, sim->cap, sim->sh, sim->kappa,
                   dt2, 2, 1, sim->g_acc, sim->pairH, sim->Dc_acc, sim->pD, sim->gdir_acc, sim->sc_dev->E + 6,
                   &sim->sc_dev->min_s, P.precision == IPC_PREC_MIXED);
    prof_end(sim, PROF_BARRIER);
    if (P.mu > 0) {
      prof_begin(sim, PROF_FRICTION);
      launch_friction(cs, S, sim->xv, sim->xv_t, sim->n_fric, sim->f_ids, sim->f_w, sim->f_n, sim->f_lam, P.mu,
                      P.eps_v * dt, dt2, 2, sim->g_acc, sim->f_Hu, sim->Dc_acc, sim->pD, sim->gdir_acc,
                      sim->sc_dev->E + 9);
      prof_end(sim, PROF_FRICTION);
    }
    if ((s = build_abd_contact(sim, P.mu > 0 ? sim->n_fric : 0))) return s;
    assembly_end(sim);
    launch_rhs(cs, ndof, sim->g, sim->gdir, sim->rhs);
    launch_dinv(cs, sim->n_nodes, S.bsr_diag, sim->Hval, sim->Dc, sim->Dinv);
    // ---- PCG
    const int fp32 = P.precision == IPC_PREC_MIXED ? 1 : 0;
    const int n_fric_it = P.mu > 0 ? sim->n_fric : 0;
    // batches: scenes whose Newton iteration has converged are left out of the solve (direction 0)
    sim->pcg_skip_on = false;
    if (sim->n_scenes > 1 && !scene_done.empty()) {
      for (int k = 0; k < sim->n_scenes; ++k) sim->pcg_skip_h[k] = scene_done[k] ? 1 : 0;
      CUDA_TRY(cudaMemcpyAsync(sim->d_pcg_skip, sim->pcg_skip_h, sizeof(int) * sim->n_scenes, cudaMemcpyHostToDevice,
                               cs));
      sim->pcg_skip_on = true;
    }
    prof_begin(sim, PROF_PCG_SETUP);
    build_incidence(sim, n_fric_it);
    if (fp32) {
      launch_to_float(cs, 144 * (size_t)sim->cap, sim->pairH, sim->pairH32, &sim->sc_dev->n_pairs, 144);
      if (n_fric_it) launch_to_float(cs, 9 * (size_t)n_fric_it, sim->f_Hu, sim->fHu32);
      launch_to_float(cs, 9 * (size_t)sim->n_nodes, sim->Dinv, sim->Dinv32);
      if (sim->nab) launch_to_float(cs, 9 * (size_t)sim->abd_cap, sim->abd_val, sim->abd_val32, sim->abd_ptr + sim->nab, 9);
    }
    if (sim->autotune_pending) {
      // time every launch shape on this system (same right-hand side, same tolerance) and keep the fastest
      const int rowgs[4] = {1, 2, 4, 8};
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      int best_r = sim->tune_rowg, best_b = sim->tune_bps;
      for (int bi = 0; bi < 2; ++bi)
        for (int ri = 0; ri < 4; ++ri) {
          sim->tune_rowg = rowgs[ri];
          sim->tune_bps = bi + 1;
          float ms = 0.f;
          if (pcg_prepare(sim, fp32) != IPC_OK) {
            // no co-resident plan with this shape (e.g. too few CTAs for the batch's scenes): not a candidate
            sim->tune_ms[4 * bi + ri] = -1.f;
            continue;
          }
          if ((s = coarse_setup(sim, fp32, n_fric_it))) return s;
          for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, cs);
            if ((s = pcg_run(sim, fp32, P.pcg_rtol, max_pcg, n_fric_it))) return s;
            cudaEventRecord(e1, cs);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
          }
          sim->tune_ms[4 * bi + ri] = ms;
          if (ms < best) { best = ms; best_r = sim->tune_rowg; best_b = sim->tune_bps; }
        }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      sim->tune_rowg = best_r;
      sim->tune_bps = best_b;
      sim->autotune_pending = false;
    }
    // the partition follows the contact work at the first Newton iteration of a step, when the coarse level
    // (whose aggregates are the CTA row segments) is rebuilt anyway
    if ((s = pcg_prepare(sim, fp32, it == 0 && P.coarse_rebuild <= 0))) return s;
    // the coarse level is rebuilt at the first Newton iteration of a step when the launch shape changed,
    // when it failed or is missing, after coarse_rebuild steps (every step by default), or when the
    // previous step needed 30 % more PCG iterations per solve than the step it was built in
    const int keep = P.coarse_rebuild;
    if (keep < 0 && !(it == 0 && sim->co_built_this_step)) {
      // rebuilt at every Newton iteration
      if ((s = coarse_setup(sim, fp32, n_fric_it))) return s;
      sim->co_built_this_step = true;
    } else if (it == 0 && !sim->co_built_this_step) {
      const bool stale = sim->co_plan_stamp != sim->plan_stamp || !sim->co_ok || sim->co_force_rebuild ||
                         sim->co_steps_since_build >= std::max(keep, 1) ||
                         (sim->co_iters_ref > 0.0 && sim->co_last_step_avg > 1.3 * sim->co_iters_ref);
      if (stale) {
        if ((s = coarse_setup(sim, fp32, n_fric_it))) return s;
        sim->co_steps_since_build = 0;
        sim->co_iters_ref = 0.0;
      }
      sim->co_built_this_step = true;
    } else if (sim->co_plan_stamp != sim->plan_stamp || sim->co_force_rebuild) {
      if ((s = coarse_setup(sim, fp32, n_fric_it))) return s;
      sim->co_steps_since_build = 0;
      sim->co_iters_ref = 0.0;
    }
    prof_end(sim, PROF_PCG_SETUP);
    prof_begin(sim, PROF_PCG);
    const long long fb0 = sim->pcg_fallbacks, fbi0 = sim->pcg_fallback_iters;
    if ((s = pcg_run(sim, fp32, P.pcg_rtol, max_pcg, n_fric_it))) return s;
    sim->pcg_skip_on = false;
    prof_end(sim, PROF_PCG);
    // ---- direction norms and CCD bound
    launch_pnorm(cs, ndof, sim->p, nk3, sim->pD, sim->sc_dev->pn);
    if (sim->n_scenes > 1) launch_pnorm_scenes(cs, S, ndof, sim->p, nk3, sim->pD);
    launch_vertex_disp(cs, S, sim->p, sim->pD, sim->pv);
    prof_begin(sim, PROF_CCD);
    if (sweep) {
      // one traversal: the CCD bound and the candidates of the line search and the next iterate
      CUDA_TRY(cudaMemsetAsync(&sim->sc_dev->n_cand, 0, sizeof(int), cs));
      launch_sweep_bvh(cs, S, sim->xv, sim->pv, sim->bvh_pad, P.s_ccd, ACCD_MAX_ITER, sim->tri_tree, sim->edge_tree,
                       sim->cand, &sim->sc_dev->n_cand, sim->ccap, &sim->sc_dev->alpha, &sim->sc_dev->n_ccd,
                       &sim->sc_dev->flags);
    } else {
      ccd(sim, sim->xv, sim->pv);
    }
    prof_end(sim, PROF_CCD);
    if ((s = sync_scalars(sim))) return s;
    CUDA_TRY(cudaGetLastError());
    const ipcsim::Scal& h = *sim->sc_host;
    // smallest squared distance of every scene's iterate (for the adaptive stiffness)
    std::vector<double> s_it(sim->n_scenes, bits_to_double(h.min_s));
    if (sim->n_scenes > 1)
      for (int k = 0; k < sim->n_scenes; ++k) s_it[k] = bits_to_double(sim->min_sc_h[k]);
    if (h.flags & ERRF_BVH) return finish(IPC_ERR_BVH_OVERFLOW, "BVH traversal stack overflow");
    if (h.flags & ERRF_ACC) return finish(IPC_ERR_NAN, "an energy, gradient or Hessian term is not finite or exceeds 2^94");
    if (h.flags & ERRF_INC) return finish(IPC_ERR_CUDA, "contact incidence list overflow");
    if (h.flags & ERRF_ABD) {
      // the ABD coupling list overflowed: grow it and redo this iteration
      if ((s = grow_abd_list(sim, 4 * sim->abd_cap))) return finish(s, "ABD coupling list growth failed");
      continue;
    }
    if (h.n_pairs > sim->cap) {
      if ((s = grow_pairs(sim, h.n_pairs))) {
        const std::string m = sim->err;
        return finish(s, m.c_str());
      }
      rec_current = false;
      continue;
    }
    if (sweep && h.n_cand > sim->ccap) {
      if ((s = grow_cand(sim, h.n_cand))) {
        const std::string m = sim->err;
        return finish(s, m.c_str());
      }
      continue;
    }
    sim->cand_valid = sweep;
    ++it;
    st.newton_iters = it;
    st.pcg_iters_total += h.pcg_out[0] + (int)(sim->pcg_fallback_iters - fbi0);
    st.pcg_fallbacks += (int)(sim->pcg_fallbacks - fb0);
    if (sim->prof) {
      sim->pcg_iters_acc += h.pcg_out[0];
      sim->pcg_pair_iters_acc += (long long)h.pcg_out[0] * std::min(h.n_pairs, sim->cap);
      sim->pcg_fric_iters_acc += (long long)h.pcg_out[0] * (P.mu > 0 ? sim->n_fric : 0);
    }
    st.pcg_iters_max = std::max(st.pcg_iters_max, h.pcg_out[0]);
    sim->co_step_iters += h.pcg_out[0];
    ++sim->co_step_solves;
    if (h.pcg_out[1] == 3) ++st.pcg_unconverged;
    st.n_pairs_max = std::max(st.n_pairs_max, h.n_pairs);
    st.n_ccd_max = std::max(st.n_ccd_max, h.n_ccd);
    double E = total_energy(sim, sim->E_h);
    if (!std::isfinite(E)) return finish(IPC_ERR_NAN, "non-finite energy");
    if (h.pcg_out[1] == 2) return finish(IPC_ERR_NAN, "non-finite PCG iterate");
    if (h.pcg_out[1] == 1) return finish(IPC_ERR_PCG, "PCG breakdown (p^T A p <= 0)");
    double pn = bits_to_double(h.pn[0]), pdn = bits_to_double(h.pn[1]);
    if (!std::isfinite(pn)) return finish(IPC_ERR_NAN, "non-finite Newton direction");
    double min_s_it = bits_to_double(h.min_s);
    if (min_s_it < 1e299) st.min_dist = std::min(st.min_dist, std::sqrt(min_s_it));
    st.pnorm_end = pn / (dt * sim->L);
    st.energy_end = E;
    if (sim->n_scenes > 1) {
      // ---- batches: every scene has its own convergence test, CCD bound and line search, so each
      //      advances as it would alone (pairs never cross scenes, the energy is a sum over scenes)
      const int ns = sim->n_scenes;
      if (scene_done.empty()) scene_done.assign(ns, 0);
      std::vector<double> al(ns, 0.0), E0(ns), pns(ns), pds(ns);
      std::vector<char> need_test(ns, 0);
      bool all_done = true;
      for (int k = 0; k < ns; ++k) {
        E0[k] = total_energy(sim, sim->E_sc_v.data() + 8 * k);
        pns[k] = bits_to_double(sim->pn_sc_h[2 * k]);
        pds[k] = bits_to_double(sim->pn_sc_h[2 * k + 1]);
        if (!scene_done[k] && pds[k] == 0.0 && pns[k] <= tol_abs) scene_done[k] = 1;
        if (scene_done[k]) continue;
        all_done = false;
        al[k] = std::min(1.0, bits_to_double(sim->alpha_sc_h[k]));
        need_test[k] = pds[k] == 0.0;  // while kinematic targets are not reached the CCD-feasible step is taken
      }
      if (all_done) { converged = true; break; }
      int halv = 0;
      for (;;) {
        CUDA_TRY(cudaMemcpyAsync(sim->alpha_trial_dev, al.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, cs));
        launch_trial_scenes(cs, S, ndof, nk3, sim->z, sim->p, sim->z_trial, sim->xk, sim->pD, sim->xk_hat,
                            sim->xk_trial);
        double E_tot = 0;
        if ((s = energy_at(sim, sim->z_trial, sim->xk_trial, sim->xv_trial, &E_tot, nullptr))) return s;
        bool changed = false, pending = false;
        for (int k = 0; k < ns; ++k) {
          if (!need_test[k]) continue;
          const double Ek = total_energy(sim, sim->E_sc_v.data() + 8 * k);
          if (Ek <= E0[k] + 1e-13 * std::fabs(E0[k])) { need_test[k] = 0; continue; }
          al[k] *= 0.5;
          changed = true;
          // no decrease resolvable above rounding within the tolerance: this scene is stationary
          if (al[k] * pns[k] <= tol_abs) { al[k] = 0.0; need_test[k] = 0; scene_done[k] = 1; continue; }
          pending = true;
        }
        if (changed) ++halv;
        if (!pending) {
          if (changed) {
            // steps changed after the last evaluation: place every scene at its final step
            CUDA_TRY(cudaMemcpyAsync(sim->alpha_trial_dev, al.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, cs));
            launch_trial_scenes(cs, S, ndof, nk3, sim->z, sim->p, sim->z_trial, sim->xk, sim->pD, sim->xk_hat,
                                sim->xk_trial);
            launch_vertex_positions(cs, S, sim->z_trial, sim->xk_trial, sim->xv_trial);
            active_set(sim, sim->xv_trial);
          }
          break;
        }
        if (halv > 40) return finish(IPC_ERR_LS_STALL, "line search stalled");
      }
      st.ls_halvings += halv;
      for (int k = 0; k < ns; ++k)
        if (!scene_done[k] || al[k] > 0.0) st.alpha_min = std::min(st.alpha_min, al[k]);
      rec_current = true;  // the active set at the accepted trial
      std::swap(sim->z, sim->z_trial);
      std::swap(sim->xk, sim->xk_trial);
      sim->cand_valid = false;
      if ((s = adapt_kappa(sim, s_it, &scene_done))) return s;
      bool all = true;
      for (int k = 0; k < ns; ++k) all = all && scene_done[k];
      if (all) { converged = true; break; }
      continue;
    }
    bool dirichlet_done = (pdn == 0.0);
    if (dirichlet_done && pn <= tol_abs) { converged = true; break; }
    double alpha = std::min(1.0, bits_to_double(h.alpha));
    double E_new = 0;
    if (dirichlet_done) {
      int halv = 0;
      bool stationary = false;
      for (;;) {
        launch_trial(cs, ndof, nk3, sim->z, sim->p, alpha, sim->z_trial, sim->xk, sim->pD, sim->xk_hat, sim->xk_trial);
        if ((s = energy_at(sim, sim->z_trial, sim->xk_trial, sim->xv_trial, &E_new, nullptr))) return s;
        if (E_new <= E + 1e-13 * std::fabs(E)) break;
        alpha *= 0.5;
        ++halv;
        // no decrease resolvable above rounding within the tolerance: the iterate is stationary
        if (alpha * pn <= tol_abs) { stationary = true; break; }
        if (halv > 40) return finish(IPC_ERR_LS_STALL, "line search stalled");
      }
      st.ls_halvings += halv;
      if (stationary) { converged = true; break; }
      rec_current = true;  // the accepted trial is the last one evaluated
    } else {
      launch_trial(cs, ndof, nk3, sim->z, sim->p, alpha, sim->z_trial, sim->xk, sim->pD, sim->xk_hat, sim->xk_trial);
      launch_vertex_positions(cs, S, sim->z_trial, sim->xk_trial, sim->xv_trial);
      active_set(sim, sim->xv_trial);
      rec_current = true;
    }
    st.alpha_min = std::min(st.alpha_min, alpha);
    std::swap(sim->z, sim->z_trial);
    std::swap(sim->xk, sim->xk_trial);
    sim->cand_valid = false;
    if ((s = adapt_kappa(sim, s_it, nullptr))) return s;
  }
  if (!converged) return finish(IPC_ERR_NEWTON_MAXIT, "Newton did not converge");
  CUDA_TRY(cudaGetLastError());
  // PCG iterations per solve of this step, for the coarse level's rebuild policy
  if (sim->co_step_solves > 0) {
    sim->co_last_step_avg = (double)sim->co_step_iters / sim->co_step_solves;
    if (sim->co_iters_ref == 0.0) sim->co_iters_ref = sim->co_last_step_avg;
  }
  ++sim->co_steps_since_build;
  launch_velocity(cs, ndof, sim->z, sim->z_t, 1.0 / dt, sim->zd);
  CUDA_TRY(cudaStreamSynchronize(cs));
  CUDA_TRY(cudaGetLastError());
  std::memcpy(sim->h_Tcur.data(), kin_T_next, sizeof(double) * 12 * sim->nkb);
  return IPC_OK;
}

}  // namespace

extern "C" {

ipc_status sim_step(ipcsim* sim, const double* kin_T_next, ipc_step_stats* stats) {
  if (!sim) return IPC_ERR_ARG;
  if (sim->nkb && !kin_T_next) { sim->err = "kinematic transforms required"; return IPC_ERR_ARG; }
  for (int i = 0; i < 12 * sim->nkb; ++i)
    if (!std::isfinite(kin_T_next[i])) {
      sim->err = "non-finite kinematic transform (body " + std::to_string(i / 12) + ")";
      if (stats) { *stats = ipc_step_stats{}; stats->status = IPC_ERR_ARG; }
      return IPC_ERR_ARG;
    }
  ipc_step_stats st{};
  st.alpha_min = 1.0;
  st.min_dist = 1e300;
  bool started = false;
  const ipc_status code = step_body(sim, kin_T_next, st, started);
  st.status = code;
  if (code != IPC_OK && started) {
    // any failure after the start of the step: back to the state at its start (x_t, v_t unchanged, and the
    // barrier stiffness of the step's start)
    const int ndof = 3 * sim->n_nodes, nk3 = 3 * sim->nk;
    cudaMemcpyAsync(sim->z, sim->z_t, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, sim->st);
    if (nk3) cudaMemcpyAsync(sim->xk, sim->xk_t, sizeof(double) * nk3, cudaMemcpyDeviceToDevice, sim->st);
    if (sim->kappa_cur != sim->kappa_step) {
      sim->kappa_cur = sim->kappa_step;
      sim->kappa = sim->kappa_cur[0];
      cudaMemcpyAsync(sim->d_scene_kappa, sim->kappa_cur.data(), sizeof(double) * sim->n_scenes,
                      cudaMemcpyHostToDevice, sim->st);
    }
    cudaStreamSynchronize(sim->st);
  }
  st.kappa_end = sim->kappa_cur.empty() ? sim->kappa : sim->kappa_cur[0];
  if (stats) *stats = st;
  return code;
}

ipc_status sim_step_many(ipcsim* const* sims, int n, const double* const* kin_T_next_host, ipc_step_stats* stats_host,
                         ipc_status* status_host) {
  if (n < 0 || (n && !sims)) return IPC_ERR_ARG;
  std::vector<ipc_status> st(n, IPC_OK);
  std::vector<std::thread> th;
  th.reserve(n);
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      cudaSetDevice(dev);
      st[i] = sim_step(sims[i], kin_T_next_host ? kin_T_next_host[i] : nullptr, stats_host ? stats_host + i : nullptr);
    });
  for (auto& t : th) t.join();
  ipc_status worst = IPC_OK;
  for (int i = 0; i < n; ++i) {
    if (status_host) status_host[i] = st[i];
    if (st[i] != IPC_OK && worst == IPC_OK) worst = st[i];
  }
  return worst;
}

ipc_status sim_set_kinematic(ipcsim* sim, const double* kin_T_host) {
  if (!sim || (sim->nkb && !kin_T_host)) return IPC_ERR_ARG;
  if (!sim->nkb) return IPC_OK;
  CUDA_TRY(cudaMemcpyAsync(sim->T_dev, kin_T_host, sizeof(double) * 12 * sim->nkb, cudaMemcpyHostToDevice, sim->st));
  launch_kin_targets(sim->st, sim->S, sim->T_dev, sim->xk, sim->stitch_hat);
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  std::memcpy(sim->h_Tcur.data(), kin_T_host, sizeof(double) * 12 * sim->nkb);
  return IPC_OK;
}

ipc_status sim_set_params(ipcsim* sim, const double* logE_host, double mu) {
  if (!sim) return IPC_ERR_ARG;
  if (logE_host) {
    int nt = sim->nt;
    std::vector<double> m(nt), l(nt);
    for (int e = 0; e < nt; ++e) {
      double E = std::exp(logE_host[e]), nu = sim->h_nu[e];
      if (!std::isfinite(E)) { sim->err = "non-finite Young's modulus"; return IPC_ERR_ARG; }
      m[e] = E / (2 * (1 + nu));
      l[e] = E * nu / ((1 + nu) * (1 - 2 * nu)) + m[e];
    }
    sim->h_logE.assign(logE_host, logE_host + nt);
    if (nt) {
      CUDA_TRY(cudaMemcpyAsync(sim->d_mu, m.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, sim->st));
      CUDA_TRY(cudaMemcpyAsync(sim->d_lam, l.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, sim->st));
      CUDA_TRY(cudaStreamSynchronize(sim->st));
    }
  }
  if (mu >= 0) {
    if (mu > 0 && sim->fcap == 0) {
      ipc_status s = grow_fric(sim, 1024);
      if (s) return s;
    }
    sim->P.mu = mu;
  }
  return IPC_OK;
}

ipc_status sim_set_joint_targets(ipcsim* sim, const double* vec_b_host, const double* t_host) {
  if (!sim) return IPC_ERR_ARG;
  const int nj = sim->nj;
  for (const double* h : {vec_b_host, t_host})
    if (h)
      for (int i = 0; i < 3 * nj; ++i)
        if (!std::isfinite(h[i])) { sim->err = "non-finite joint target"; return IPC_ERR_ARG; }
  if (nj == 0) return IPC_OK;
  if (vec_b_host) CUDA_TRY(cudaMemcpyAsync(sim->jt_vb, vec_b_host, sizeof(double) * 3 * nj, cudaMemcpyHostToDevice, sim->st));
  if (t_host) CUDA_TRY(cudaMemcpyAsync(sim->jt_t, t_host, sizeof(double) * 3 * nj, cudaMemcpyHostToDevice, sim->st));
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  return IPC_OK;
}

ipc_status sim_adjoint(ipcsim* sim, const double* z_t, const double* zd_t, const double* z_next,
                       const double* kin_T_t_host, const double* kin_T_next_host, const double* gz_next,
                       const double* gzd_next, double* gz_t, double* gzd_t, double* glogE, double* gmu_host) {
  if (!sim || !z_t || !zd_t || !z_next || !gz_next || !gzd_next || !gz_t || !gzd_t) return IPC_ERR_ARG;
  if (sim->nkb && (!kin_T_t_host || !kin_T_next_host)) { sim->err = "kinematic transforms required"; return IPC_ERR_ARG; }
  if (sim->P.kappa_adaptive) {
    sim->err = "sim_adjoint needs a fixed barrier stiffness (kappa_adaptive is on)";
    return IPC_ERR_ARG;
  }
  const DevScene& S = sim->S;
  const ipc_params& P = sim->P;
  cudaStream_t cs = sim->st;
  const int ndof = 3 * sim->n_nodes, nk3 = 3 * sim->nk;
  const double dt = P.dt, dt2 = dt * dt;
  ipc_status s;
  // kinematic positions at t and t+1
  if (sim->nkb) {
    CUDA_TRY(cudaMemcpyAsync(sim->T_dev, kin_T_t_host, sizeof(double) * 12 * sim->nkb, cudaMemcpyHostToDevice, cs));
    launch_kin_targets(cs, S, sim->T_dev, sim->xk_t, sim->stitch_hat);
    CUDA_TRY(cudaStreamSynchronize(cs));
    CUDA_TRY(cudaMemcpyAsync(sim->T_dev, kin_T_next_host, sizeof(double) * 12 * sim->nkb, cudaMemcpyHostToDevice, cs));
  }
  launch_kin_targets(cs, S, sim->T_dev, sim->xk_hat, sim->stitch_hat);
  launch_predict(cs, S, z_t, zd_t, dt, sim->grav, sim->z_t, sim->z_tilde);
  launch_vertex_positions(cs, S, z_t, sim->xk_t, sim->xv_t);
  rebuild_trees(sim, sim->xv_t);
  // friction lag at x_t
  sim->n_fric = 0;
  if (P.mu > 0) {
    for (;;) {
      CUDA_TRY(cudaMemsetAsync(sim->sc_dev, 0, sizeof(ipcsim::Scal), cs));
      cull(sim, sim->xv_t);
      if ((s = sync_scalars(sim))) return s;
      if (sim->sc_host->n_pairs > sim->cap) { if ((s = grow_pairs(sim, sim->sc_host->n_pairs))) return s; continue; }
      break;
    }
    int n = sim->sc_host->n_pairs;
    if (n > sim->fcap && (s = grow_fric(sim, n))) return s;
    launch_friction_lag(cs, pair_grid(sim->cap), S, sim->xv_t, sim->rec, &sim->sc_dev->n_pairs, sim->cap, sim->sh,
                        sim->kappa, sim->f_ids, sim->f_w, sim->f_n, sim->f_lam, sim->f_rec);
    sim->n_fric = n;
  }
  // unprojected Hessian at z*
  launch_vertex_positions(cs, S, z_next, sim->xk_hat, sim->xv);
  for (;;) {
    CUDA_TRY(cudaMemsetAsync(sim->sc_dev, 0, sizeof(ipcsim::Scal), cs));
    if ((s = assembly_begin(sim))) return s;
    if (nk3) CUDA_TRY(cudaMemsetAsync(sim->pD, 0, sizeof(double) * nk3, cs));
    cull(sim, sim->xv);
    launch_elastic_assembly(cs, S, sim->xv, dt2, 0, sim->g_acc, sim->Hconst, sim->Hval, sim->sc_dev->E + 3, 0,
                            sim->el_tU, sim->el_tG);
    launch_abd_orth(cs, S, z_next, P.kappa_A, dt2, 2, 0, sim->g_acc, sim->H_acc, sim->sc_dev->E + 15);
    launch_joints(cs, S, z_next, dt2, 2, sim->g_acc, sim->H_acc, sim->sc_dev->E + 18);
    launch_barrier(cs, pair_grid(sim->cap), S, sim->xv, sim->rec, &sim->sc_dev->n_pairs, sim->cap, sim->sh,
                   sim->kappa, dt2, 2, 0, sim->g_acc, sim->pairH, sim->Dc_acc, sim->pD, sim->gdir_acc,
                   sim->sc_dev->E + 6, nullptr);
    if (P.mu > 0)
      launch_friction(cs, S, sim->xv, sim->xv_t, sim->n_fric, sim->f_ids, sim->f_w, sim->f_n, sim->f_lam, P.mu,
                      P.eps_v * dt, dt2, 2, sim->g_acc, sim->f_Hu, sim->Dc_acc, sim->pD, sim->gdir_acc,
                      sim->sc_dev->E + 9);
    if ((s = sync_scalars(sim))) return s;
    if (sim->sc_host->flags & ERRF_BVH) { sim->err = "BVH traversal stack overflow"; return IPC_ERR_BVH_OVERFLOW; }
    if (sim->sc_host->n_pairs > sim->cap) { if ((s = grow_pairs(sim, sim->sc_host->n_pairs))) return s; continue; }
    break;
  }
  for (int tries = 0;; ++tries) {
    // the ABD coupling list of the unprojected Hessian (grown until it fits)
    CUDA_TRY(cudaMemsetAsync(&sim->sc_dev->flags, 0, sizeof(int), cs));
    if (tries > 0) {
      // a retry: rebuild the ABD blocks without the partial contact blocks of the overflowed pass (the
      // gradient accumulated again is not used by the adjoint; the FEM blocks hold no contact terms)
      CUDA_TRY(cudaMemsetAsync(sim->H_acc + 27 * (size_t)sim->nfb, 0, sizeof(acc_t) * 27 * (size_t)(sim->nnzb - sim->nfb),
                               cs));
      launch_abd_orth(cs, S, z_next, P.kappa_A, dt2, 2, 0, sim->g_acc, sim->H_acc, sim->sc_dev->E + 15);
      launch_joints(cs, S, z_next, dt2, 2, sim->g_acc, sim->H_acc, sim->sc_dev->E + 18);
    }
    if ((s = build_abd_contact(sim, P.mu > 0 ? sim->n_fric : 0))) return s;
    if ((s = sync_scalars(sim))) return s;
    if (!(sim->sc_host->flags & ERRF_ABD)) break;
    if (tries > 8 || (s = grow_abd_list(sim, 4 * sim->abd_cap))) { sim->err = "ABD coupling list growth failed"; return IPC_ERR_CAPACITY; }
  }
  assembly_end(sim);
  launch_dinv(cs, sim->n_nodes, S.bsr_diag, sim->Hval, sim->Dc, sim->Dinv);
  launch_axpy(cs, ndof, gz_next, 1.0 / dt, gzd_next, sim->rhs);
  {
    const int n_fric_adj = P.mu > 0 ? sim->n_fric : 0;
    build_incidence(sim, n_fric_adj);
    if ((s = pcg_prepare(sim, 0))) return s;
    if ((s = coarse_setup(sim, 0, n_fric_adj))) return s;
    // rtol 1e-12 on the unprojected (possibly indefinite) Hessian: more true-residual restarts than a
    // Newton solve, and a two-level solve that spent them above 1e-10 is repeated with block Jacobi alone
    const int max_it = 10 * ndof + 1000;
    sim->pcg_max_replace = 40;
    s = pcg_run(sim, 0, 1e-12, max_it, n_fric_adj);
    if (!s && sim->co_ok) {
      ipcsim::Scal* h = sim->sc_host;
      if (cudaMemcpyAsync(h->pcg_out, sim->sc_dev->pcg_out, sizeof(h->pcg_out), cudaMemcpyDeviceToHost, cs) ||
          cudaMemcpyAsync(&h->pcg_res, &sim->sc_dev->pcg_res, sizeof(double), cudaMemcpyDeviceToHost, cs) ||
          cudaStreamSynchronize(cs)) {
        s = IPC_ERR_CUDA;
        sim->err = "adjoint PCG status copy failed";
      } else if (h->pcg_out[1] == 3 && !(h->pcg_res <= 1e-10)) {
        ++sim->pcg_fallbacks;
        s = pcg_launch(sim, 0, 1e-12, max_it, n_fric_adj, false);
      }
    }
    sim->pcg_max_replace = 10;
    if (s) return s;
    // the coarse level now belongs to this adjoint's Hessian: the next step builds its own
    sim->co_steps_since_build = 1 << 20;
  }
  // contractions with lam (= sim->p)
  if (glogE) launch_theta_grad(cs, S, sim->xv, sim->p, dt2, glogE);
  double* tmp = sim->y;  // scratch: friction gradient, then M lam
  CUDA_TRY(cudaMemsetAsync(sim->sc_dev->E + 18, 0, 6 * sizeof(acc_t), cs));
  if (P.mu > 0 && sim->n_fric) {
    CUDA_TRY(cudaMemsetAsync(sim->g_acc, 0, sizeof(acc_t) * 3 * ndof, cs));
    launch_friction(cs, S, sim->xv, sim->xv_t, sim->n_fric, sim->f_ids, sim->f_w, sim->f_n, sim->f_lam, P.mu,
                    P.eps_v * dt, dt2, 1, sim->g_acc, nullptr, nullptr, nullptr, nullptr, sim->sc_dev->E + 21);
    launch_acc_finalize(cs, ndof, sim->g_acc, nullptr, tmp);
    launch_dot(cs, ndof, tmp, sim->p, sim->sc_dev->E + 18);
  }
  launch_mass_apply(cs, S, sim->p, dt, tmp, gzd_t);
  launch_axpy(cs, ndof, tmp, -1.0 / dt, gzd_next, gz_t);
  if (P.mu > 0) {
    CUDA_TRY(cudaMemsetAsync(sim->gz_acc, 0, sizeof(acc_t) * 3 * ndof, cs));
    launch_friction_apply(cs, S, sim->n_fric, sim->f_ids, sim->f_w, sim->f_Hu, sim->p, sim->gz_acc);
    // through the lagged normal forces, normals and closest points at x_t
    launch_friction_lag_adjoint(cs, S, sim->xv, sim->xv_t, sim->n_fric, sim->f_ids, sim->f_rec, sim->sh, P.mu,
                                P.eps_v * dt, dt2, sim->p, sim->gz_acc);
    launch_acc_finalize(cs, ndof, sim->gz_acc, gz_t, gz_t);
  }
  if ((s = sync_scalars(sim))) return s;
  CUDA_TRY(cudaGetLastError());
  if (sim->sc_host->pcg_out[1] == 3 && !(sim->sc_host->pcg_res <= 1e-10)) {
    char buf[32];
    snprintf(buf, sizeof buf, "%.3e", sim->sc_host->pcg_res);
    sim->err = std::string("adjoint PCG stopped at relative residual ") + buf;
    return IPC_ERR_PCG;
  }
  if (sim->sc_host->pcg_out[1] == 3) sim->sc_host->pcg_out[1] = 0;
  if (sim->sc_host->pcg_out[1]) { sim->err = "adjoint PCG breakdown (Hessian not positive definite)"; return IPC_ERR_PCG; }
  if (gmu_host && P.mu > 0) *gmu_host += -sim->E_h[6] / P.mu;
  return IPC_OK;
}

ipc_status sim_tuning(ipcsim* sim, int rowg, int blocks_per_sm, int autotune_next_step, int* out4, float* ms8) {
  if (!sim) return IPC_ERR_ARG;
  if (rowg > 0) {
    if (rowg != 1 && rowg != 2 && rowg != 4 && rowg != 8) { sim->err = "rowg must be 1, 2, 4 or 8"; return IPC_ERR_ARG; }
    sim->tune_rowg = rowg;
  }
  if (blocks_per_sm > 0) sim->tune_bps = std::min(blocks_per_sm, 4);
  if (autotune_next_step) sim->autotune_pending = true;
  if (out4) {
    out4[0] = sim->tune_rowg;
    out4[1] = sim->tune_bps;
    out4[2] = sim->plan.grid;
    out4[3] = sim->plan_resident ? 1 : 0;
  }
  if (ms8) std::memcpy(ms8, sim->tune_ms, sizeof(sim->tune_ms));
  return IPC_OK;
}

ipc_status sim_coarse_info(const ipcsim* sim, long long* out4) {
  if (!sim || !out4) return IPC_ERR_ARG;
  out4[0] = sim->co.n_agg;
  out4[1] = sim->co.n_solves;
  out4[2] = sim->co.n_max;
  out4[3] = sim->co_ok ? 1 : 0;
  return IPC_OK;
}

ipc_status sim_pcg_residency(ipcsim* sim, int streamed) {
  if (!sim) return IPC_ERR_ARG;
  sim->pcg_streamed = streamed != 0;
  return IPC_OK;
}

ipc_status sim_profile(ipcsim* sim, int enable) {
  if (!sim) return IPC_ERR_ARG;
  sim->prof = enable != 0;
  if (enable != 1) return IPC_OK;  // pause (0) or resume (2): keep what has been accumulated
  for (int k = 0; k < 8; ++k) { sim->prof_ms[k] = 0; sim->prof_n[k] = 0; sim->ev_open[k] = false; }
  sim->pcg_iters_acc = sim->pcg_pair_iters_acc = sim->pcg_fric_iters_acc = 0;
  return IPC_OK;
}

ipc_status sim_profile_read(const ipcsim* sim, double* ms8, long long* n8, long long* work4) {
  if (!sim) return IPC_ERR_ARG;
  for (int k = 0; k < 8; ++k) {
    if (ms8) ms8[k] = sim->prof_ms[k];
    if (n8) n8[k] = sim->prof_n[k];
  }
  if (work4) {
    work4[0] = sim->pcg_iters_acc;
    work4[1] = sim->pcg_pair_iters_acc;
    work4[2] = sim->pcg_fric_iters_acc;
    work4[3] = sim->nnzb;
  }
  return IPC_OK;
}

ipc_status sim_get_state(const ipcsim* csim, double* x, double* v, double* q, double* qd, int on_device) {
  ipcsim* sim = const_cast<ipcsim*>(csim);
  if (!sim) return IPC_ERR_ARG;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  size_t nfb = sizeof(double) * 3 * sim->nf, nab = sizeof(double) * 12 * sim->nab;
  if (x && nfb) CUDA_TRY(cudaMemcpyAsync(x, sim->z, nfb, k, sim->st));
  if (v && nfb) CUDA_TRY(cudaMemcpyAsync(v, sim->zd, nfb, k, sim->st));
  if (q && nab) CUDA_TRY(cudaMemcpyAsync(q, sim->z + 3 * sim->nf, nab, k, sim->st));
  if (qd && nab) CUDA_TRY(cudaMemcpyAsync(qd, sim->zd + 3 * sim->nf, nab, k, sim->st));
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  return IPC_OK;
}

ipc_status sim_positions(const ipcsim* csim, double* xv_dev) {
  ipcsim* sim = const_cast<ipcsim*>(csim);
  if (!sim || !xv_dev) return IPC_ERR_ARG;
  launch_vertex_positions(sim->st, sim->S, sim->z, sim->xk, xv_dev);
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

ipc_status sim_set_state(ipcsim* sim, const double* x, const double* v, const double* q, const double* qd,
                         int on_device) {
  if (!sim) return IPC_ERR_ARG;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  size_t nfb = sizeof(double) * 3 * sim->nf, nab = sizeof(double) * 12 * sim->nab;
  if (x && nfb) CUDA_TRY(cudaMemcpyAsync(sim->z, x, nfb, k, sim->st));
  if (v && nfb) CUDA_TRY(cudaMemcpyAsync(sim->zd, v, nfb, k, sim->st));
  if (q && nab) CUDA_TRY(cudaMemcpyAsync(sim->z + 3 * sim->nf, q, nab, k, sim->st));
  if (qd && nab) CUDA_TRY(cudaMemcpyAsync(sim->zd + 3 * sim->nf, qd, nab, k, sim->st));
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  return IPC_OK;
}

// ---------------------------------------------------------------------------
// stage entry points
// ---------------------------------------------------------------------------

ipc_status sim_eval_elastic(ipcsim* sim, const double* x_dev, int project, double* E_dev, double* grad_dev,
                            double* H_dev) {
  if (!sim || !x_dev || !E_dev || !grad_dev) return IPC_ERR_ARG;
  // the simulator's gradient accumulators and its scratch energy slot 7
  acc_t* Eacc = sim->sc_dev->E + 21;
  CUDA_TRY(cudaMemsetAsync(Eacc, 0, 3 * sizeof(acc_t), sim->st));
  CUDA_TRY(cudaMemsetAsync(sim->g_acc, 0, sizeof(acc_t) * 9 * (size_t)sim->nf, sim->st));
  launch_elastic(sim->st, sim->S, x_dev, 1.0, H_dev ? 2 : 1, project, sim->g_acc, H_dev, Eacc);
  launch_acc_finalize(sim->st, 3 * (size_t)sim->nf, sim->g_acc, nullptr, grad_dev);
  launch_acc_finalize(sim->st, 1, Eacc, nullptr, E_dev);
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  CUDA_TRY(cudaGetLastError());
  return IPC_OK;
}

ipc_status sim_active_pairs(ipcsim* sim, const double* x_dev, int cap, int* rec_dev, double* s_dev, int* n_host) {
  if (!sim || !x_dev || !rec_dev || !n_host || cap < 0) return IPC_ERR_ARG;
  ipc_status so = grow_order(sim, cap);
  if (so) return so;
  CUDA_TRY(cudaMemsetAsync(&sim->sc_dev->flags, 0, sizeof(int), sim->st));
  rebuild_trees(sim, x_dev);
  cull_into(sim, x_dev, rec_dev, s_dev, cap);
  CUDA_TRY(cudaMemcpyAsync(n_host, &sim->sc_dev->n_pairs, sizeof(int), cudaMemcpyDeviceToHost, sim->st));
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  CUDA_TRY(cudaGetLastError());
  return *n_host > cap ? IPC_ERR_CAPACITY : IPC_OK;
}

ipc_status sim_eval_barrier(ipcsim* sim, const double* x_dev, int n, const int* rec_dev, int project, double* E_dev,
                            double* grad_dev, double* H_dev) {
  if (!sim || !x_dev || n < 0 || (n && !rec_dev) || !E_dev || !grad_dev || (n && !H_dev)) return IPC_ERR_ARG;
  int* n_dev;
  double* pDz;
  acc_t *Dc, *gdir, *gnode, *Eacc;
  ipc_status s;
  const size_t n3 = 3 * (size_t)sim->n_nodes;
  if ((s = dalloc(sim, &n_dev, 1))) return s;
  if ((s = dalloc(sim, &Dc, 27 * (size_t)sim->n_nodes))) return s;
  if ((s = dalloc(sim, &gdir, 3 * n3))) return s;
  if ((s = dalloc(sim, &pDz, 3 * (size_t)std::max(sim->nk, 1)))) return s;
  if ((s = dalloc(sim, &gnode, 3 * n3))) return s;
  if ((s = dalloc(sim, &Eacc, 3))) return s;
  CUDA_TRY(cudaMemcpyAsync(n_dev, &n, sizeof(int), cudaMemcpyHostToDevice, sim->st));
  CUDA_TRY(cudaMemsetAsync(Dc, 0, sizeof(acc_t) * 27 * (size_t)sim->n_nodes, sim->st));
  CUDA_TRY(cudaMemsetAsync(gdir, 0, sizeof(acc_t) * 3 * n3, sim->st));
  CUDA_TRY(cudaMemsetAsync(pDz, 0, sizeof(double) * 3 * (size_t)std::max(sim->nk, 1), sim->st));
  CUDA_TRY(cudaMemsetAsync(gnode, 0, sizeof(acc_t) * 3 * n3, sim->st));
  CUDA_TRY(cudaMemsetAsync(Eacc, 0, sizeof(acc_t) * 3, sim->st));
  launch_barrier(sim->st, pair_grid(n), sim->S, x_dev, rec_dev, n_dev, n, sim->sh, sim->kappa, 1.0, 2, project, gnode,
                 H_dev, Dc, pDz, gdir, Eacc, nullptr);
  launch_acc_finalize(sim->st, n3, gnode, nullptr, grad_dev);
  launch_acc_finalize(sim->st, 1, Eacc, nullptr, E_dev);
  CUDA_TRY(cudaStreamSynchronize(sim->st));
  CUDA_TRY(cudaGetLastError());
  dfree(sim, n_dev); dfree(sim, Dc); dfree(sim, gdir); dfree(sim, pDz); dfree(sim, gnode); dfree(sim, Eacc);
  return IPC_OK;
}

ipc_status sim_pcg_partition(const int* row, int nf, int nab, int grid, const int* node_scene, int n_scenes,
                             const int* row_extra, int* out4, int* seg, int* abd_seg, int* cta_scene) {
  if (!row || !out4 || !seg || !abd_seg || !cta_scene || nf < 0 || nab < 0 || grid < 2 || n_scenes < 1 ||
      (n_scenes > 1 && !node_scene))
    return IPC_ERR_ARG;
  const int n_rows = nf + 4 * nab;
  std::vector<int> r(row, row + n_rows + 1), ns;
  if (node_scene) ns.assign(node_scene, node_scene + n_rows);
  std::vector<int> extra;
  if (row_extra) extra.assign(row_extra, row_extra + nf);
  PcgPlan P;
  pcg_plan_rows(r, nf, nab, grid, ns, n_scenes, P, row_extra ? &extra : nullptr);
  out4[0] = P.n_fem_ctas;
  out4[1] = P.n_abd_ctas;
  out4[2] = P.n_psc;
  out4[3] = P.max_rows;
  for (int c = 0; c <= P.n_fem_ctas; ++c) seg[c] = P.seg[c];
  for (int c = 0; c <= P.n_abd_ctas; ++c) abd_seg[c] = P.abd_seg[c];
  for (int c = 0; c < grid; ++c) cta_scene[c] = P.cta_scene[c];
  return IPC_OK;
}

ipc_status sim_ccd_alpha(ipcsim* sim, const double* x_dev, const double* p_dev, double* alpha_host, int* n_cand_host) {
  if (!sim || !x_dev || !p_dev || !alpha_host) return IPC_ERR_ARG;
  unsigned long long one = double_bits(1.0);
  CUDA_TRY(cudaMemcpyAsync(&sim->sc_dev->alpha, &one, sizeof(one), cudaMemcpyHostToDevice, sim->st));
  if (sim->n_scenes > 1) {
    const std::vector<unsigned long long> ones(sim->n_scenes, one);
    CUDA_TRY(cudaMemcpyAsync(sim->alpha_sc_dev, ones.data(), sizeof(one) * ones.size(), cudaMemcpyHostToDevice,
                             sim->st));
    CUDA_TRY(cudaStreamSynchronize(sim->st));  // the staging vector goes out of scope
  }
  CUDA_TRY(cudaMemsetAsync(&sim->sc_dev->n_ccd, 0, sizeof(int), sim->st));
  CUDA_TRY(cudaMemsetAsync(&sim->sc_dev->flags, 0, sizeof(int), sim->st));
  rebuild_trees(sim, x_dev);
  ccd(sim, x_dev, p_dev);
  if (sync_scalars(sim)) return IPC_ERR_CUDA;
  if (sim->sc_host->flags & ERRF_BVH) { sim->err = "BVH traversal stack overflow"; return IPC_ERR_BVH_OVERFLOW; }
  CUDA_TRY(cudaGetLastError());
  *alpha_host = bits_to_double(sim->sc_host->alpha);
  if (n_cand_host) *n_cand_host = sim->sc_host->n_ccd;
  return IPC_OK;
}

}  // extern "C"
