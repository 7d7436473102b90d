// Host-side launchers of the ipcsim kernels (declarations).
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include "bvh.cuh"
#include "common.cuh"

namespace ipc {

// Device memory of one simulator: from the caller's allocator when one was
// given at creation (e.g. PyTorch's caching allocator), else from cudaMalloc.
struct DevAlloc {
  void* (*alloc_fn)(size_t, void*, void*) = nullptr;
  void (*free_fn)(void*, void*, void*) = nullptr;
  void* ctx = nullptr;
  cudaStream_t st = nullptr;
  long long by_allocator = 0, direct = 0, bytes = 0;
  cudaError_t get(void** p, size_t nbytes) {
    *p = nullptr;
    if (alloc_fn) {
      *p = alloc_fn(nbytes, (void*)st, ctx);
      if (!*p) return cudaErrorMemoryAllocation;
      ++by_allocator;
    } else {
      cudaError_t e = cudaMalloc(p, nbytes);
      if (e != cudaSuccess) return e;
      ++direct;
    }
    bytes += (long long)nbytes;
    return cudaSuccess;
  }
  void put(void* p, size_t nbytes) {
    if (!p) return;
    if (free_fn) free_fn(p, (void*)st, ctx);
    else cudaFree(p);
    bytes -= (long long)nbytes;
  }
};

// Streaming multiprocessors of the current device (looked up once per device).
int device_sms();
// Blocks of a grid-stride launch over n items, `per_block` items per block and
// at most `per_sm` resident blocks per SM of the current device (at least 1).
inline int stride_grid(long long n, int per_block, int per_sm) {
  const long long want = (n + per_block - 1) / per_block, cap = (long long)device_sms() * per_sm;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// Kernel launches issued by this library (all simulators, all threads).
extern unsigned long long g_kernel_launches;
inline void count_launch(int n = 1) { __atomic_fetch_add(&g_kernel_launches, (unsigned long long)n, __ATOMIC_RELAXED); }

// Gather descriptor of one contact pair (barrier pairs at [0, cap), friction
// pairs at [cap, cap + fcap)): for every slot the first node of its vertex (-1:
// kinematic or zero weight) and, for ABD vertices (bit j of abd), the rest
// position that weights the body's pseudo-nodes 1..3.
struct __align__(16) PairDesc {
  int node[4];
  int abd;
  int pad[3];
  double xb[4][3];
};

// Coarse level of the PCG preconditioner (coarse.cu): an aggregate is the
// row segments of a run of consecutive FEM CTAs of one solve (so that a
// solve's coarse size stays bounded), six rigid-body modes each.
struct CoarseDev {
  const float* inv32 = nullptr;   // per solve: dense (P^T A P)^-1 in FP32, row-major n_s x n_s at off[s];
                                  // null: no coarse level
  const double* inv64 = nullptr;  // the same in FP64; when set, the FP64 solver applies it in FP64 (tight
                                  // tolerances: an FP32 coarse product is not a fixed linear operator)
  const long long* off = nullptr; // (solves)
  const int* solve_lo = nullptr;  // (solves) first aggregate of every solve
  const int* solve_n = nullptr;   // (solves) coarse unknowns of every solve (6 per aggregate)
  const int* cta_agg = nullptr;   // (FEM CTAs) aggregate of every FEM CTA, -1 none
  const int* agg_cta = nullptr;   // (aggregates, 2) FEM CTAs [first, end) of every aggregate
  const double* centre = nullptr; // (aggregates, 3)
  const double* rot = nullptr;    // (aggregates) 1 / RMS radius scaling the rotations, 0: none
  const double* x = nullptr;      // (nf, 3) positions the modes are built at
  double* part = nullptr;         // (FEM CTAs, 6) every CTA's part of P^T v for the current iteration
  int smem_off = -1;              // byte offset in the dynamic shared memory where every CTA stages its
                                  // aggregate's six rows of the inverse once per solve; -1: read from global
};
// host-side layout of the coarse level for one PCG plan
struct CoarseLayout {
  int n_agg = 0, n_solves = 0, n_max = 0, n_ctas = 0, group = 1;
  long long total = 0, total_n = 0;
  bool consecutive = true;
  std::vector<int> node_agg, agg_solve, solve_lo, solve_n, cta_agg, agg_cta;
  std::vector<long long> off, boff;
};
// the same on the device
struct CoarseDevLayout {
  int n_agg = 0, n_solves = 0, n_max = 0;
  long long total = 0, total_n = 0;
  const int* node_agg = nullptr;
  const int* agg_solve = nullptr;
  const int* solve_lo = nullptr;
  const int* solve_n = nullptr;
  const int* agg_cta = nullptr;    // (aggregates, 2) FEM CTAs [first, end) of every aggregate
  const long long* off = nullptr;
  const long long* boff = nullptr;
};
// largest coarse size of one solve: runs of CTAs are merged into aggregates until it holds
constexpr int COARSE_MAX_UNKNOWNS = 768;

// Arguments of one PCG solve (see pcg.cu).  CTAs [0, n_fem_ctas) own the FEM
// rows seg_row[c] .. seg_row[c + 1]; the others own ABD bodies
// b = cta - n_fem_ctas (mod n_abd_ctas).  Pointers of the operator type
// (double, or float when fp32) are passed as void*.
struct PcgArgs {
  DevScene S;
  int n_nodes;
  int n_fem_ctas, n_abd_ctas;
  const int* seg_row;        // (n_fem_ctas + 1)
  int resident;              // stage each FEM CTA's operator rows in shared memory
  const int* row;
  const int* col;
  const void* op;            // BSR values in the CTA-major plane layout, operator type
  const void* dinv;          // (n_nodes, 9) preconditioner blocks, operator type
  const double* val64;       // BSR values as assembled (FP64), for the true residual
  const void* pairH;         // (cap, 144) barrier pair blocks, operator type
  const void* fHu;           // (n_fric, 9) friction blocks, operator type
  const double* pairH64;
  const double* fHu64;
  const int* rec;
  const int* n_pairs;        // device count of active pairs
  int cap;
  int n_fric;
  const int* f_ids;
  const double* f_w;
  const PairDesc* desc;      // (cap + fcap) gather descriptors of the pairs
  const int* inc_ptr;        // (nf + nab + 1) contact incidences per owner
  const int2* inc;           // (code, owner) ordered by owner; code = pair << 3 | friction << 2 | slot
  int max_rows;              // most FEM rows of one CTA
  int acc_doubles;           // doubles of shared memory reserved for the row products
  const int* abd_ptr;        // (nab + 1) contact coupling blocks per ABD body
  const int* abd_ent;        // column node << 2 | pseudo-node row
  const double* abd_val;     // (entries, 9)
  const float* abd_val32;    // FP32 copy (mixed precision)
  long long abd_cap;
  const double* b;
  double* x;
  void* vec;                 // nine FP64 vectors of 3 n_nodes values
  double* t64;               // 3 n_nodes FP64 scratch (true residual)
  void* partial;             // pcg_partial_doubles(grid) doubles
  double rtol;
  int max_iter;
  int max_replace;           // true-residual restarts before the solve gives up (<= 0: 10)
  int fp32;
  int* out;                  // [iterations, status, true-residual restarts]
  double* res;               // [relative residual]
  long long inc_cap;         // entries of inc
  int* check;                // non-null: validate every gathered index, record the first bad site here, skip it
  // independent solves (a batch of scenes): every CTA serves the rows of one scene, each scene runs
  // its own recurrences, tolerance and stop; n_psc = 1 is one solve over all CTAs
  int n_psc;
  const int* abd_seg;        // (n_abd_ctas + 1) ABD bodies of every ABD CTA
  const int* cta_scene;      // (grid) scene of every CTA, -1 for a CTA without rows
  const int* sc_ptr;         // (n_psc + 1) CTAs of every scene, in sc_cta
  const int* sc_cta;
  const int* scene_skip;     // (n_psc) or null: nonzero = scene not solved (x = 0)
  double* sc_res;            // (n_psc) or null: relative residual of every scene
  int* sc_it;                // (n_psc) or null: iterations of every scene
  CoarseDev co;              // coarse level of the preconditioner (co.inv null: block Jacobi only)
};

// Row partition of one PCG launch shape.
struct PcgPlan {
  int grid = 0, n_fem_ctas = 0, n_abd_ctas = 0;
  std::vector<int> seg;      // FEM CTA row boundaries, then nf + 4 b for every ABD body
  std::vector<int> abd_seg;  // ABD body boundaries of the ABD CTAs
  int n_psc = 1;             // independent solves
  std::vector<int> cta_scene, sc_ptr, sc_cta;
  int max_rows = 0, max_blocks = 0;
  int acc_doubles = 0;       // row products in shared memory: 3 per FEM row, 12 per ABD body of a CTA
};


// fem.cu
void launch_predict(cudaStream_t, const DevScene&, const double* z, const double* zd, double dt, const double* g,
                    double* z_t, double* z_tilde);
void launch_kin_targets(cudaStream_t, const DevScene&, const double* T, double* xk_hat, double* stitch_hat);
void launch_vertex_positions(cudaStream_t, const DevScene&, const double* z, const double* xk, double* xv);
void launch_vertex_disp(cudaStream_t, const DevScene&, const double* p, const double* pD, double* pv);
// Accumulating outputs (acc_t: three words per value, see common.cuh): g (n_nodes, 3), Hval (nnzb, 9),
// Dc (n_nodes, 9), gdir (n_nodes, 3) and E (one value) are added into, never overwritten.
void launch_inertia(cudaStream_t, const DevScene&, const double* z, const double* z_tilde, acc_t* g, acc_t* E,
                    int want_grad);
// hess_fp32: the projected Hessian in FP32 (mixed precision); energy and gradient stay FP64
void launch_elastic(cudaStream_t, const DevScene&, const double* xv, double scale, int mode, int project, acc_t* g,
                    double* tetH, acc_t* E, int hess_fp32 = 0);
// The Newton assembly of the elastic term: gradient into g, and the FEM BSR blocks written as
// Hval = Hconst + the tets' blocks (gathered in tet order from the per-tet scratch tU (78 nt), tG (12 nt))
void launch_elastic_assembly(cudaStream_t, const DevScene&, const double* xv, double scale, int project, acc_t* g,
                             const double* Hconst, double* Hval, acc_t* E, int hess_fp32, double* tU, double* tG);
void launch_stitch(cudaStream_t, const DevScene&, const double* xv, const double* stitch_hat, double k_c, double scale,
                   int mode, acc_t* g, acc_t* E);
void launch_abd_orth(cudaStream_t, const DevScene&, const double* z, double kappa_A, double scale, int mode, int project,
                     acc_t* g, acc_t* Hval, acc_t* E);
void launch_joints(cudaStream_t, const DevScene&, const double* z, double scale, int mode, acc_t* g, acc_t* Hval,
                   acc_t* E);
// out[i] = (base ? base[i] : 0) + the value of accumulator i, for i < n
void launch_acc_finalize(cudaStream_t, size_t n, const acc_t* acc, const double* base, double* out);
void launch_trial(cudaStream_t, int ndof, int nk3, const double* z, const double* p, double alpha, double* z_out,
                  const double* xk, const double* pD, const double* xk_hat, double* xk_out);
void launch_velocity(cudaStream_t, int ndof, const double* z, const double* z_t, double inv_dt, double* zd);
void launch_pnorm(cudaStream_t, int ndof, const double* p, int nk3, const double* pD, unsigned long long* out);
// batches: per-scene max |p_F|, |p_D| into S.pn_sc; trial step with the step of each scene (S.alpha_trial)
void launch_pnorm_scenes(cudaStream_t, const DevScene& S, int ndof, const double* p, int nk3, const double* pD);
void launch_trial_scenes(cudaStream_t, const DevScene& S, int ndof, int nk3, const double* z, const double* p,
                         double* z_out, const double* xk, const double* pD, const double* xk_hat, double* xk_out);
void launch_sub(cudaStream_t, int n, const double* a, const double* b, double* o);

// contact.cu
void launch_barrier(cudaStream_t, int grid, const DevScene&, const double* xv, const int* rec, const int* n_dev, int cap,
                    double sh, double kappa, double scale, int mode, int project, acc_t* g, double* pairH, acc_t* Dc,
                    const double* pD, acc_t* gdir, acc_t* E, unsigned long long* min_s, int hess_fp32 = 0);
// f_rec (may be null): (kind, type, primitive a, primitive b) of every friction pair, for the adjoint
void launch_friction_lag(cudaStream_t, int grid, const DevScene&, const double* xv, const int* rec, const int* n_dev,
                         int cap, double sh, double kappa, int* f_ids, double* f_w, double* f_n, double* f_lam,
                         int* f_rec = nullptr);
// adjoint: -scale d(lam . grad D)/dx_t through the lagged friction data, added into gz (DOF space)
void launch_friction_lag_adjoint(cudaStream_t, const DevScene&, const double* xv, const double* xv_t, int n,
                                 const int* f_ids, const int* f_rec, double sh, double mu, double eps, double scale,
                                 const double* lam_dof, acc_t* gz);
void launch_friction(cudaStream_t, const DevScene&, const double* xv, const double* xv_t, int n, const int* f_ids,
                     const double* f_w, const double* f_n, const double* f_lam, double mu, double eps, double scale,
                     int mode, acc_t* g, double* f_Hu, acc_t* Dc, const double* pD, acc_t* gdir, acc_t* E);

// order.cu: canonical order of atomically appended lists (stable LSD radix sort of 64-bit keys with an
// index payload; the length min(*n_dev, cap) is read on the device)
struct OrderWork {
  unsigned long long *keys = nullptr, *keys_tmp = nullptr;  // (cap)
  int *idx = nullptr, *idx_tmp = nullptr;                   // (cap)
  int* hist = nullptr;                                      // sort_hist_ints(cap)
  int* tiles = nullptr;                                     // scan_tile_ints(sort_hist_ints(cap))
  int* rec_tmp = nullptr;                                   // (cap, 8)
  double* s_tmp = nullptr;                                  // (cap)
  int cap = 0;
};
size_t sort_hist_ints(int cap);
void launch_sort_u64(cudaStream_t, const int* n_dev, int cap, int key_bits, unsigned long long* keys, int* idx,
                     unsigned long long* keys_tmp, int* idx_tmp, int* hist, int* scan_tiles);
// contact pairs (and their squared distances, may be null) into (kind, a, b) order; prim_bits >= the bits of
// every primitive id
void launch_sort_pairs(cudaStream_t, const int* n_dev, int cap, int prim_bits, int* rec, double* rec_s,
                       const OrderWork& W);

// cull.cu
void launch_cull_brute(cudaStream_t, const DevScene&, const double* xv, double sh, int* rec, double* rec_s, int* count,
                       int cap);
void launch_ccd_brute(cudaStream_t, const DevScene&, const double* xv, const double* pv, double s_frac, int max_iter,
                      unsigned long long* alpha_bits, int* n_cand);

// bvh.cu
cudaError_t bvh_alloc(Bvh& B, int n, DevAlloc& mem);
void bvh_free(Bvh& B, DevAlloc& mem);
void bvh_leaf_boxes(cudaStream_t, Bvh& B, const int* ids, int nvp, const double* xv, const double* pv, double pad);
void bvh_refit(cudaStream_t, Bvh& B);
void bvh_build(cudaStream_t, Bvh& B);
void launch_cull_bvh(cudaStream_t, const DevScene&, const double* xv, double sh, double pad, Bvh& tri, Bvh& edge,
                     int* rec, double* rec_s, int* count, int cap, int* err);
void launch_ccd_bvh(cudaStream_t, const DevScene&, const double* xv, const double* pv, double s_frac, int max_iter,
                    Bvh& tri, Bvh& edge, unsigned long long* alpha_bits, int* n_cand, int* err);
void bvh_rebuild(cudaStream_t, const DevScene&, const double* xv, double pad, Bvh& tri, Bvh& edge);
void launch_sweep_bvh(cudaStream_t, const DevScene&, const double* xv, const double* pv, double pad, double s_frac,
                      int max_iter, Bvh& tri, Bvh& edge, int* cand, int* n_cand, int ccap,
                      unsigned long long* alpha_bits, int* n_ccd, int* err);
void launch_filter_active(cudaStream_t, int grid, const DevScene&, const double* xv, double sh, const int* cand,
                          const int* n_cand, int ccap, int* rec, double* rec_s, int* count, int cap);

// adjoint.cu
void launch_theta_grad(cudaStream_t, const DevScene&, const double* xv, const double* lam, double scale, double* out);
void launch_mass_apply(cudaStream_t, const DevScene&, const double* lam, double dt, double* y, double* yd);
void launch_friction_apply(cudaStream_t, const DevScene&, int n, const int* f_ids, const double* f_w, const double* f_Hu,
                           const double* lam, acc_t* y);
// out: an accumulator (three words)
void launch_dot(cudaStream_t, int n, const double* a, const double* b, acc_t* out);
void launch_axpy(cudaStream_t, int n, const double* x, double alpha, const double* y, double* out);

// exclusive scan of n ints in place (tiles: scan_tile_ints(n) ints of scratch)
size_t scan_tile_ints(size_t n);
void launch_scan_exclusive(cudaStream_t, int n, int* a, int* tiles);

// pcg.cu
void launch_dinv(cudaStream_t, int n_nodes, const int* diag, const double* val, const double* Dc, double* Dinv);
void launch_rhs(cudaStream_t, int n, const double* g, const double* gdir, double* rhs);
constexpr int PCG_ROW_GROUP = 4;  // default threads per FEM row in the PCG
constexpr int PCG_REPLICA_COUNT = 8;
constexpr int PCG_SCENES_MAX = 256;  // independent solves of one launch (one decision thread each)
// Contact work of a FEM row in units of a stored BSR block, per contact incidence (a 3 x 12 pair-block row
// times the pair's vertices is about four blocks' work): the FEM rows are partitioned with it at the first
// Newton iteration of every step (the plan then stays for the step; the coarse level is rebuilt at that
// iteration anyway).  Two simulators stepping concurrently once disagreed with sequential stepping when
// the plan followed the contacts at every iteration; that was the process-wide shared-memory limit race
// (fixed), not the partition.
constexpr int PCG_CONTACT_WEIGHT = 4;
inline size_t pcg_partial_doubles(int grid) { return (size_t)PCG_REPLICA_COUNT * 7 * grid; }
// co-resident CTAs of the PCG kernel for this shape (rowg: threads per FEM row, 1, 2, 4 or 8)
int pcg_max_blocks(int threads, int fp32, int rowg, size_t dyn_smem);
size_t pcg_smem_limit();
// node_scene (empty: one solve) gives the scene of every row; scenes get CTAs of their own when their rows
// are contiguous and the grid has room, else the plan is one solve
void pcg_plan_rows(const std::vector<int>& row, int nf, int nab, int grid, const std::vector<int>& node_scene,
                   int n_scenes, PcgPlan& P, const std::vector<int>* row_extra = nullptr);
// dynamic shared memory of a PCG CTA: contact sums of its rows, plus the operator rows when resident
size_t pcg_contact_bytes(const PcgPlan& P);
size_t pcg_resident_bytes(const PcgPlan& P, int fp32);
cudaError_t launch_pcg(cudaStream_t, int grid, int threads, const PcgArgs& a, int rowg, size_t dyn_smem);
void launch_layout(cudaStream_t, int n_seg, const int* seg, const int* row, const double* src, void* dst, int fp32);
void launch_incidence(cudaStream_t, const DevScene& S, const int* rec, const int* n_pairs, int cap, int n_fric,
                      const int* f_ids, const double* f_w, int* inc_ptr, int* cursor, int* tiles, int2* inc,
                      long long inc_cap, PairDesc* desc, int* err);
// Work of the per-body coupling lists' order, sized for 4 (pair capacity + friction pairs) chunk slots.
struct AbdChunks {
  unsigned long long *keys = nullptr, *keys_tmp = nullptr;
  int *idx = nullptr, *idx_tmp = nullptr, *hist = nullptr, *tiles = nullptr;
  int *size = nullptr, *scan = nullptr, *pos = nullptr;
  int* n = nullptr;        // chunk slots of the current lists (device)
  int pair_bits = 1, key_bits = 1;
  int cap = 0;
  // the raw lists (one entry per pair and slot) and the merge of equal codes, sized like the lists
  int* ent_raw = nullptr;
  double* val_raw = nullptr;
  unsigned long long *ekeys = nullptr, *ekeys_tmp = nullptr;
  int *eidx = nullptr, *eidx_tmp = nullptr, *ehist = nullptr, *etiles = nullptr, *ehead = nullptr;
  int* body_cnt = nullptr;  // (n_abd + 1)
  int code_bits = 1, ekey_bits = 1;
  long long ecap = 0;
};
void launch_abd_contact(cudaStream_t, const DevScene& S, const int* rec, const int* n_pairs, int cap,
                        const double* pairH, int n_fric, const int* f_ids, const double* f_w, const double* f_Hu,
                        int* abd_ptr, const AbdChunks& C, int* ent, double* entv, long long ent_cap, acc_t* Hval,
                        acc_t* Dc, int* err);
void launch_to_float(cudaStream_t, size_t n, const double* src, float* dst, const int* n_dev = nullptr, int stride = 0);

// coarse.cu: layout of the coarse level for a plan, and its build (aggregate centres, Galerkin matrix
// P^T A P per solve, Gauss-Jordan inversion); status (solves): nonzero where a pivot failed
void coarse_layout(const PcgPlan& P, int nf, CoarseLayout& L);
cudaError_t launch_coarse_build(cudaStream_t, const DevScene& S, const CoarseDevLayout& D, const int* seg,
                                const double* x, const double* val, const int* rec, const int* n_pairs, int cap,
                                const double* pairH, int n_fric, const int* f_ids, const double* f_w,
                                const double* f_Hu, double* Ac, acc_t* Ac_acc, double* centre, double* rot,
                                double* gj_buf, int* status);

// conservative-advancement iterations per CCD candidate
constexpr int ACCD_MAX_ITER = 10000;

}  // namespace ipc
