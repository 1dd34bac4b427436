// Device-side data structures and kernel launchers of the hz library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace hz {

// One supernode of a batched multifrontal factorisation (56 bytes).
// widest merged solve supernode of the complex128 sweeps (see FactorDev::ssn)
constexpr int kMaxSolveK = 448;
constexpr int kMaxSolveK64 = 512;   // the same for the complex64 sweeps

struct SnDev {
  int32_t k, m, first, parent;   // pivots, front order, first vector index, parent (-1 root)
  int32_t ld, pad_;              // panel leading dimension (m, or m rounded up to 4 for complex64)
  int64_t rowoff;                // into rowlist / cptr slots
  int64_t paneloff;              // panel (m x k, column-major, ld m) in the factor store
  int64_t uoff;                  // update vector (m - k) in the solve workspace
  int64_t frontoff;              // front (m x m, column-major) in the frontal workspace
};

// Device view of a batched symbolic factorisation plus its numeric factor.
struct FactorDev {
  int nmat = 0, nsn = 0, nlev = 0;
  int32_t maxk = 0, maxm = 0;
  int32_t bwd_rows = 512;        // rows per backward partial task (<= 512)
  int64_t ntot = 0, nrows = 0, panel_elems = 0, u_elems = 0, front_elems = 0, nentries = 0;
  SnDev* sn = nullptr;
  // single-right-hand-side sweeps: supernodes of the solve tree, in which chains of
  // supernodes (each the only child of the next, with nested row sets) are merged into one
  // solve supernode whose panel (appended after the factor panels, panel_elems onwards)
  // holds the inverse of the merged unit lower diagonal block and the matching off-diagonal
  // block; equal to sn where nothing is merged.  snlev: levels of the solve tree.
  SnDev* ssn = nullptr;
  int snlev = 0;
  int64_t solve_panel_elems = 0;      // panel_elems plus the merged solve panels
  // merge steps, in order: the solve supernode's panel (offset, ld = its rows), its width
  // so far w, and the appended original supernode's panel (offset, ld, k_s, m_s); and the
  // scratch for one step's k_s x w block
  struct MergeStep {
    int64_t moff, soff;
    int32_t ldm, w, lds, ks, ms;
  };
  std::vector<MergeStep> merges;
  int64_t merge_tmp_elems = 0;
  void* merge_tmp = nullptr;
  int32_t* rowlist = nullptr;
  int64_t* cptr = nullptr;
  int64_t* cidx = nullptr;
  int32_t* rel = nullptr;
  int64_t* reloff = nullptr;
  int32_t* gidx = nullptr;       // ntot: global index of each local vector entry
  // gather-form prolongation: per global dof, its local entries and weights
  int64_t nglob = 0;
  int64_t* pptr = nullptr;
  int32_t* pidx = nullptr;
  double* pw = nullptr;
  // frequency-free entry values and their front positions
  int64_t* epos = nullptr;
  double* ek = nullptr;
  double2* em = nullptr;
  double2* eb = nullptr;
  // task arrays (device) and per-level host offsets
  int2* fwd_tasks = nullptr;     // (sn, row block)
  int4* bwd_tasks = nullptr;     // (sn, col block, row chunk, global bfin index): partial sums
  int4* bfin_tasks = nullptr;    // (sn, col block, first partial task of its level, chunks), all levels
  unsigned int* bwd_counters = nullptr;  // one per bfin task: partial-sum CTAs done (reset by the last)
  void* bwd_partial = nullptr;   // 32 values per backward partial task (max over levels)
  int2* ea_tasks = nullptr;      // (child sn, col block)
  int2* wg_tasks = nullptr;      // (sn, row block of the off-diagonal part)
  int4* cb_tasks = nullptr;      // (sn, row tile, col tile, scratch-relative offset unused)
  int4* tc_tasks = nullptr;      // complex64 path: (sn, 128-row tile, 128-col tile, 0), tensor-core Schur update
  int64_t* h_tc_ptr = nullptr;   // nlev + 1 (host)
  int64_t* scr_off = nullptr;    // per supernode: offset of its W block in the level scratch
  int32_t* lev_sn = nullptr;
  int64_t* h_lev_ptr = nullptr;       // nlev + 1 (host)
  int64_t* h_fwd_ptr = nullptr;       // nlev + 1
  int64_t* h_bwd_ptr = nullptr;
  int64_t* h_bfin_ptr = nullptr;
  int64_t* h_wg_ptr = nullptr;
  int64_t* h_cb_ptr = nullptr;
  int64_t* h_ea_ptr = nullptr;        // nlev * maxslot + 1, grouped (level, slot)
  int64_t* h_ent_ptr = nullptr;       // nlev + 1: entries of each level's fronts
  // factorisation groups (whole matrices, one after the other in one frontal workspace):
  // per level (and slot) the start of each group's tasks, groups + 1 entries each
  int32_t ngrp = 1;
  int64_t *h_lev_g = nullptr, *h_ent_g = nullptr, *h_wg_g = nullptr, *h_cb_g = nullptr, *h_tc_g = nullptr;
  int64_t* h_ea_g = nullptr;          // ((level * max_slot + slot) * (groups + 1) + group)
  cudaEvent_t* level_events = nullptr;  // optional (diagnostics): 2 * nlev + 1 events around sweep levels
  int* h_fwd_rt = nullptr;            // nlev: complex128 forward task rows (16 or 64)
  int* h_bwd_rows = nullptr;          // nlev: complex128 backward chunk rows
  int32_t max_slot = 0;
  // kernel variants of the schedule (host-side counts, reported through hz_stats)
  int32_t v_fwd_wide = 0, v_fwd_narrow = 0, v_bwd_wide = 0, v_bwd_narrow = 0;
  int64_t v_bwd_split = 0, v_tc_tiles = 0, v_tc_multi = 0;
  int32_t v_tc_kstages = 0, v_max_k = 0;
  int32_t tc_wait = 1 << 22;          // polls of the first wait on a tensor-core completion barrier
  // the assembly tree on the host (levels, supernode widths and heights), from which the
  // sweep task lists can be rebuilt (sweep autotuner)
  std::vector<int32_t> t_lev_ptr, t_lev_sn, t_sn_k, t_sn_m;
  int32_t sweep_chunk = 0;            // rows of a wide backward chunk in use
  double sweep_scale = 1.0;           // scale of the narrow-level task threshold in use
  int64_t scratch_elems = 0;          // max over levels of sum (m-k) k
  // algorithmic cost of one forward+backward sweep (host-side)
  double solve_bytes = 0, solve_flops = 0;
  double gather_bytes = 0, prolong_bytes = 0;
  int64_t prolong_nnz = 0;
  // numeric
  int precision = 0;                  // 0: complex128, 1: complex64
  void* panels = nullptr;             // factor store
  // batched (S right-hand sides) sweep tasks and workspaces, built when block_size > 1
  int32_t mS = 0;
  int2* mfwd_tasks = nullptr;
  int4* mbwd_tasks = nullptr;
  int4* mbfin_tasks = nullptr;
  unsigned int* mbwd_counters = nullptr;
  int64_t* h_mfwd_ptr = nullptr;
  int64_t* h_mbwd_ptr = nullptr;
  int32_t mbwd_rows = 128;
  void* mt_loc = nullptr;
  void* mz_loc = nullptr;
  void* mx_loc = nullptr;
  void* mu_ws = nullptr;
  void* mbwd_partial = nullptr;
  // solve workspaces (typed by precision)
  void* t_loc = nullptr;
  void* z_loc = nullptr;
  void* x_loc = nullptr;
  void* u_ws = nullptr;
};

// Status word written by device code (pivot health).
// Column offsets of the S slots of a pseudo-block solve (negative: empty slot).
struct SlotCols {
  int64_t o[16];
};

// Per-slot operands of the slot-batched CGS2 passes (ncols < 0: empty slot).
struct SlotCgs {
  const double2* V[16];       // the slot's basis, column-major, leading dimension n
  double2* w[16];
  const double2* h[16];       // coefficients of the update pass
  int ncols[16];
};

// Per-slot Givens update: slot i's arrays at fixed strides from these bases (j < 0: skip).
struct SlotGivens {
  int m;
  int j[16];
  double2 *H, *sn, *g;
  double* cs;
  const double2 *h1, *h2, *nrm;    // S x 65 each
  double* scal;                    // S x 8: estimate, 1 / h_{j+1,j}, ..., |b| at 4
  int* brk;
};

struct SlotScale {
  const double2* w[16];
  const double* s[16];
  double2* out[16];                // null: empty slot
};

// One point source's right-hand side: at most 10 basis functions (P2 tetrahedron).
struct PointRhs {
  int64_t idx[10];
  double val[10];
  int cnt;
};

struct DevStatus {
  unsigned int zero_pivot;
  unsigned int timeout;          // a bounded wait on a tensor-core completion barrier ran out
  double min_pivot;   // stored as the bit pattern of a non-negative double (atomicMin on u64)
};

// ---- launchers (kernels.cu) -------------------------------------------------
long long launch_count();
void add_launches(long long n);   // kernels replayed inside a CUDA graph launch
void launch_fill_values(int64_t nnz, const double* K, const double2* M, const double2* B, double w,
                        double2* out, cudaStream_t st);
// One assembly-tree level: zero and fill its fronts (A_i(omega) entries), extend-add the
// children, factor, and copy the panels to the factor store.
void launch_factor_level(const FactorDev& F, int lev, int grp, double w, void* fronts, void* scratch,
                         DevStatus* status, double tiny, cudaStream_t st);

void launch_gather(const FactorDev& F, const double2* src, cudaStream_t st);
void launch_solve(const FactorDev& F, cudaStream_t st);
// Builds the merged solve panels from the factor panels (after the last factor level).
void launch_merge_panels(const FactorDev& F, cudaStream_t st);
void launch_prolong(const FactorDev& F, const double2* y, double2* z, cudaStream_t st);

void launch_local_multi(const FactorDev& F, int S, const double2* src, const double2* y, double2* dst,
                        cudaStream_t st);
void launch_interleave(int64_t n, int S, const SlotCols& off, const double2* base, double2* inter, cudaStream_t st);
void launch_deinterleave(int64_t n, int S, const SlotCols& off, const double2* inter, double2* base, cudaStream_t st);
void launch_point_rhs(const PointRhs& p, double2* out, cudaStream_t st);
void launch_interleave_put(int64_t n, int S, int i, const double2* col, double2* inter, cudaStream_t st);
// out (S x 65): per slot, maxpy pass (w -= V h) and / or dot pass (V^H w, |w|^2), reduced.
void launch_cgs_slots(int64_t n, int S, const SlotCgs& p, bool maxpy, bool dots, double2* partial, double2* out,
                      cudaStream_t st);
void launch_givens_slots(int S, const SlotGivens& p, cudaStream_t st);
void launch_scale_slots(int64_t n, int S, const SlotScale& p, cudaStream_t st);
void launch_spmv_multi(int64_t n, int S, const int64_t* rp, const int32_t* ci, const double2* val, const double2* x,
                       const double2* sub, double2* y, cudaStream_t st);
void launch_spmv_real_multi(int64_t n, int S, const int64_t* rp, const int32_t* ci, const double* val,
                            const double2* x, double2* y, cudaStream_t st);
void set_spmv_lanes(int tpr);     // 2, 4, 8 or 16 lanes per row (calling thread)
void launch_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double2* val, const double2* x,
                 const double2* sub, double2* y, cudaStream_t st);
void launch_spmv_real(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, const double2* x,
                      double2* y, cudaStream_t st);
int cgs_blocks();
void launch_cgs(int64_t n, int ncols, const double2* V, int64_t ldv, const double2* h, double2* w,
                int ndot, double2* partial, cudaStream_t st);
void launch_reduce(const double2* partial, int nblk, int ncols, double2* out, cudaStream_t st);
void launch_givens(int j, int m, double2* H, double* cs, double2* sn, double2* g, const double2* h1,
                   const double2* h2, const double2* nrm, const double* bnorm, double* est, int* breakdown,
                   double* invh, cudaStream_t st, int off = 0, double2* raw_h = nullptr, double2* raw_b = nullptr,
                   int ldb = 0);
constexpr int kComboMaxCols = 80, kComboMaxOut = 16;
void launch_combo(int64_t n, int nb1, const double2* B1, int64_t ld1, int nb2, const double2* B2, int64_t ld2,
                  const double2* coef, int nout, double2* out, int64_t ldo, double sign, bool accumulate,
                  cudaStream_t st);
void launch_init_cycle(const double2* nrm2, double2* g, int m, double* invbeta, double* beta, cudaStream_t st);
void launch_scale(int64_t n, const double2* w, const double* s, double2* out, cudaStream_t st);
void launch_gemv_add(int64_t n, int k, const double2* y, const double2* Zs, int64_t ldz, double2* x, cudaStream_t st);
void launch_update_x(int64_t n, int k, const double2* H, int ldh, const double2* g, double2* y,
                     const double2* Zs, int64_t ldz, double2* x, cudaStream_t st);
void launch_add2(int n, const double2* a, const double2* b, double2* out, cudaStream_t st);
void launch_axpby_copy(int64_t n, const double2* a, double2* out, cudaStream_t st);

}  // namespace hz
