// C ABI of the hz library: context management, per-frequency factorisation and
// the right-preconditioned FGMRES(m) driver.  See include/hz.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hz.h"
#include "dev.h"
#include "engine.h"
#include "host.h"
#include "small_la.h"

using hz::cplx;

struct hz_ctx {
  std::string err;
  hz_options opt{};
  cudaStream_t st = nullptr;
  int device = 0;
  int order = 1, levels = 1, restart = 30, precision = 0, max_iter = 1000;
  hz::Mesh mesh;       // kept for point location
  hz::Dofs dofs;       // kept for point sources
  int64_t n = 0, nnz = 0, nH = 0, nnzH = 0, zeta_nnz = 0;
  // global operator
  int64_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  double* d_K = nullptr;
  double2* d_M = nullptr;
  double2* d_B = nullptr;
  double2* d_A = nullptr;
  // coarse interpolation
  int64_t *d_Zrp = nullptr, *d_Ztrp = nullptr;
  int32_t *d_Zci = nullptr, *d_Ztci = nullptr;
  double *d_Zv = nullptr, *d_Ztv = nullptr;
  hz::FactorDev loc, crs;
  double loc_max[3] = {0, 0, 0}, crs_max[3] = {0, 0, 0};
  // iterative coarse solve: E in CSR, local coarse factors, inner GMRES workspace
  int coarse_oras = 0, cmaxit = 30;
  double ctol = 1e-2;
  hz::FactorDev cloc;
  double cloc_max[3] = {0, 0, 0};
  int64_t* d_Erp = nullptr;
  int32_t* d_Eci = nullptr;
  double* d_EK = nullptr;
  double2 *d_EM = nullptr, *d_EB = nullptr, *d_E = nullptr;
  double2 *VH = nullptr, *ZH = nullptr, *wH = nullptr, *HH = nullptr, *snH = nullptr, *gH = nullptr, *yHs = nullptr;
  double *csH = nullptr, *scalH = nullptr;
  int* brkH = nullptr;
  // Krylov workspace
  double2 *V = nullptr, *Zs = nullptr, *w = nullptr, *b = nullptr, *x = nullptr, *y = nullptr, *t = nullptr;
  double2 *rH = nullptr, *yH = nullptr;
  double2 *partial = nullptr, *h1 = nullptr, *h2 = nullptr, *nrm = nullptr;
  double2 *H = nullptr, *sn = nullptr, *g = nullptr, *ysol = nullptr;
  double *cs = nullptr, *scal = nullptr;   // scal: est, invh, invbeta, beta, |b|
  // one CUDA graph per inner-iteration index j (captured on first use)
  std::vector<cudaGraphExec_t> gexec;     // index j + restart * (recycled dimension)
  std::vector<long long> gcount;
  // GCRO-DR recycling (options.recycle = rk > 0): the recycled space C sits right before
  // the Arnoldi basis, in columns [rk - rdim, rk) of Vx (V = Vx + rk n), so that [C, V]
  // is one column-major block for CGS2
  int rk = 0, rdim = 0, ckk = 0;
  double2 *Vx = nullptr, *Ux = nullptr, *Uh = nullptr, *Ctmp = nullptr, *Uxt = nullptr, *Uht = nullptr;
  double2 *Hraw = nullptr, *Braw = nullptr, *dcoef = nullptr;
  bool graphs = true;
  int spmv_lanes = 0;                      // autotuned at the first hz_factor (0: not yet)
  bool sweeps_tuned = false;               // sweep task shapes chosen (tune_sweeps)
  bool recycle_stale = false;              // recycled space kept across hz_factor, not yet re-based
  int* brk = nullptr;
  hz::DevStatus* status = nullptr;
  double* h_pin = nullptr;                 // pinned: est, invh, invbeta, beta, brk, norm
  bool factored = false;
  hz_stats stats{};
  // pseudo-block state (block_size > 1): S right-hand sides, interleaved operator blocks
  int S = 0;
  double2 *Vb = nullptr, *Zb = nullptr, *Wc = nullptr, *Bc = nullptr, *Xc = nullptr;   // per-RHS columns
  double2 *Xi = nullptr, *Yi = nullptr, *Ti = nullptr, *Wi = nullptr, *yi = nullptr;   // interleaved n x S
  double2 *rHi = nullptr, *yHi = nullptr;                                              // interleaved nH x S
  double2 *Hb = nullptr, *snb = nullptr, *gb = nullptr, *yb = nullptr;
  double *csb = nullptr, *scalb = nullptr;
  int* brkb = nullptr;
  double2 *partial_s = nullptr, *h1s = nullptr, *h2s = nullptr, *nrms = nullptr;   // slot-batched CGS2
  // block FGMRES (krylov == HZ_KRYLOV_BLOCK): coefficients of the chunked block CGS2 passes
  // (2 passes x chunks of 64 basis columns x S columns x 65) and the cycle-end Y (m S x S)
  int krylov = 0;
  double2 *hblk = nullptr, *yblk = nullptr;
  // slot engine (continuous pseudo-block FGMRES): one right-hand side per slot
  enum { SLOT_FREE = hz_engine::SLOT_FREE, SLOT_RUN = hz_engine::SLOT_RUN, SLOT_DONE = hz_engine::SLOT_DONE };
  struct Slot {
    int state = SLOT_FREE;
    int64_t tag = -1;
    double tol = 0.0, bnorm = 0.0;
    int its = 0, j = 0;               // iterations so far; position in the current cycle
    hz_rhs_info info{0, HZ_OK, 0.0};
  };
  std::vector<Slot> slots;
  // pinned host scalars: [0, 8) single-RHS loop, then per-slot scalars, flags and |b|
  enum {
    PIN_SLOT = 8,
    PIN_FLAGS = 8 + 8 * 16,
    PIN_BNORM = 8 + 8 * 16 + 16,
    PIN_CRS = 8 + 8 * 16 + 32,        // inner coarse solve: |r_H|^2, estimate, breakdown flag
    PIN_TOTAL = 8 + 8 * 16 + 36
  };
  std::vector<void*> allocs;
  std::vector<size_t> sizes;
  int64_t bytes = 0;
};

namespace {

hz_status fail(hz_ctx* c, hz_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, HZ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <typename T>
hz_status dalloc(hz_ctx* c, T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) return HZ_OK;
  const size_t bytes = size_t(count) * sizeof(T);
  if (c->opt.hbm_budget && uint64_t(c->bytes) + bytes > c->opt.hbm_budget)
    return fail(c, HZ_ERR_OOM, "allocation exceeds hbm_budget");
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  c->sizes.push_back(bytes);
  c->bytes += int64_t(bytes);
  return HZ_OK;
}

void dfree(hz_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) {
    const size_t i = size_t(it - c->allocs.begin());
    c->bytes -= int64_t(c->sizes[i]);
    c->allocs.erase(it);
    c->sizes.erase(c->sizes.begin() + i);
  }
  cudaFree(p);
}

template <typename T>
hz_status upload(hz_ctx* c, T** dst, const std::vector<T>& v) {
  hz_status s = dalloc(c, dst, int64_t(v.size()));
  if (s != HZ_OK) return s;
  if (!v.empty()) CU(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->st));
  return HZ_OK;
}

#define TRY(expr)                     \
  do {                                \
    hz_status s_ = (expr);            \
    if (s_ != HZ_OK) return s_;       \
  } while (0)

std::vector<double2> to_d2(const std::vector<cplx>& v) {
  std::vector<double2> o(v.size());
  for (size_t i = 0; i < v.size(); i++) o[i] = make_double2(v[i].real(), v[i].imag());
  return o;
}

// Device copy of a symbolic set with its task lists.
// Task shapes of the batched triangular sweeps per assembly-tree level, and the kernel
// variants they imply (host-only; shared by the device upload and hz_plan).
// Sparse tree levels get narrow tasks.  complex128 (FP64 arithmetic bound): fewer
// tasks than two per SM -> 16-row forward tasks, 64-row backward chunks, so that such a
// level reaches every SM.  complex64: fewer tasks than one resident wave (8 CTAs per
// SM) -> 64-row forward tasks and 128-row backward chunks, which shorten each task's
// serial walk over its columns and rows (the time of a latency-bound level).
// sweep_tasks (hz_options) forces wide (1) or narrow (2) shapes on every level.
struct SweepPlan {
  std::vector<int> fwd_rt, bwd_rows;   // per level: forward task rows, backward chunk rows
  int32_t fwd_wide = 0, fwd_narrow = 0, bwd_wide = 0, bwd_narrow = 0;
  int64_t bwd_split = 0, tc_tiles = 0, tc_multi = 0;
  int32_t tc_kstages = 0, max_k = 0;
};

// The assembly-tree view the sweep schedule needs (host arrays).
struct TreeView {
  int nlev;
  const int32_t *lev_ptr, *lev_sn, *sn_k, *sn_m;
};
TreeView view_of(const hz::SymbolicSet& S) {
  return TreeView{S.nlev, S.lev_ptr.data(), S.lev_sn.data(), S.sn_k.data(), S.sn_m.data()};
}

// Solve tree of a complex128 factor: chains of supernodes in which each one is the only
// child of the next and its rows below its pivots are exactly the next one's rows (same
// order, checked on the row lists) merge, up to width merge_width, into one solve supernode
// (the top separators of a nested-dissection tree form such chains).  The triangular sweeps
// then take one dependent level per merged chain instead of one per supernode.  chain_of:
// solve supernode of each supernode; chains: members bottom to top; the solve tree's levels
// (a solve supernode one above its highest child) with its widths and heights.
struct SolveTree {
  std::vector<int32_t> chain_of;
  std::vector<std::vector<int32_t>> chains;
  std::vector<int32_t> k, m, lev_ptr, lev_sn;
  int nlev = 0;
  int64_t merged_elems = 0;           // entries of the merged panels (stored beside the factor's)
  TreeView view() const { return TreeView{nlev, lev_ptr.data(), lev_sn.data(), k.data(), m.data()}; }
};

// Merge parameters of the subdomain factors: width by precision; only the sparse top
// levels (at most two supernodes per subdomain), which bounds the duplicated panel bytes.
int local_merge_width(int precision) { return precision == 1 ? hz::kMaxSolveK64 : hz::kMaxSolveK; }
int local_merge_sparse(const hz::SymbolicSet& S) { return 2 * S.nmat; }

// sparse_max > 0: a supernode joins a chain only if its factor level holds at most that
// many supernodes (the top of a batch of trees: about one separator chain per matrix).
SolveTree plan_solve_tree(const hz::SymbolicSet& S, int merge_width, int sparse_max = 0) {
  SolveTree T;
  const int ns = int(S.sn_k.size());
  static const bool off = std::getenv("HZ_NO_SOLVE_MERGE") != nullptr;
  const bool merge = merge_width > 0 && !off;
  std::vector<int32_t> nchild(ns, 0), width;
  for (int s = 0; s < ns; s++)
    if (S.sn_parent[s] >= 0) nchild[S.sn_parent[s]]++;
  T.chain_of.assign(ns, -1);
  for (int s = 0; s < ns; s++) {                     // children before parents
    if (T.chain_of[s] < 0) {
      T.chain_of[s] = int32_t(T.chains.size());
      T.chains.push_back({s});
      width.push_back(S.sn_k[s]);
    }
    const int ch = T.chain_of[s], p = S.sn_parent[s];
    if (!merge || p <= s || nchild[p] != 1 || T.chain_of[p] >= 0 || T.chains[ch].back() != s) continue;
    if (sparse_max > 0 && (S.lev_ptr[size_t(S.sn_level[s]) + 1] - S.lev_ptr[size_t(S.sn_level[s])] > sparse_max ||
                           S.lev_ptr[size_t(S.sn_level[p]) + 1] - S.lev_ptr[size_t(S.sn_level[p])] > sparse_max))
      continue;
    if (S.sn_mat[p] != S.sn_mat[s] || S.sn_m[s] - S.sn_k[s] != S.sn_m[p] ||
        S.sn_first[p] != S.sn_first[s] + S.sn_k[s] || width[size_t(ch)] + S.sn_k[p] > merge_width)
      continue;
    bool same = true;
    for (int i = 0; i < S.sn_m[p] && same; i++)
      same = S.rowlist[size_t(S.sn_rowoff[s] + S.sn_k[s] + i)] == S.rowlist[size_t(S.sn_rowoff[p] + i)];
    if (!same) continue;
    T.chain_of[p] = ch;
    T.chains[size_t(ch)].push_back(p);
    width[size_t(ch)] += S.sn_k[p];
  }
  const int nc = int(T.chains.size());
  T.k.assign(nc, 0);
  T.m.assign(nc, 0);
  std::vector<int32_t> lev(nc, 0);
  for (int c = 0; c < nc; c++) {                     // chains in order of their first member
    const std::vector<int32_t>& ch = T.chains[size_t(c)];
    T.k[size_t(c)] = width[size_t(c)];
    T.m[size_t(c)] = S.sn_m[ch.front()];
    if (ch.size() > 1) T.merged_elems += int64_t(T.m[size_t(c)]) * T.k[size_t(c)];
    const int p = S.sn_parent[ch.back()];
    if (p >= 0) {
      const int pc = T.chain_of[p];
      lev[size_t(pc)] = std::max(lev[size_t(pc)], lev[size_t(c)] + 1);
    }
  }
  for (int c = 0; c < nc; c++) T.nlev = std::max(T.nlev, lev[size_t(c)] + 1);
  if (nc == 0) T.nlev = 0;
  T.lev_ptr.assign(T.nlev + 1, 0);
  for (int c = 0; c < nc; c++) T.lev_ptr[size_t(lev[size_t(c)]) + 1]++;
  for (int l = 0; l < T.nlev; l++) T.lev_ptr[size_t(l) + 1] += T.lev_ptr[size_t(l)];
  T.lev_sn.assign(nc, 0);
  std::vector<int32_t> fill(T.lev_ptr.begin(), T.lev_ptr.end() - (T.nlev > 0 ? 1 : 0));
  for (int c = 0; c < nc; c++) T.lev_sn[size_t(fill[size_t(lev[size_t(c)])]++)] = c;
  return T;
}

// sparse_scale multiplies the task count below which a level gets narrow tasks (the
// sweep autotuner's knob; 1 = the defaults above).
SweepPlan plan_sweeps(const TreeView& S, int precision, int bwd_rows, int sweep_tasks, double sparse_scale = 1.0) {
  SweepPlan sp;
  const int nlev = S.nlev;
  const int wide = precision == 0 ? 64 : 256;
  sp.fwd_rt.assign(nlev, wide);
  sp.bwd_rows.assign(nlev, bwd_rows);
  for (int l = 0; l < nlev; l++) {
    int64_t nf = 0, nbk = 0;
    for (int32_t q = S.lev_ptr[l]; q < S.lev_ptr[l + 1]; q++) {
      const int s = S.lev_sn[q];
      nf += (S.sn_m[s] + wide - 1) / wide;
      nbk += int64_t((S.sn_k[s] + 31) / 32) * ((S.sn_m[s] + bwd_rows - 1) / bwd_rows);
    }
    const int64_t sparse = int64_t((precision == 0 ? 2 * 152 : 8 * 152) * sparse_scale);
    const bool narrow_f = sweep_tasks == 2 || (sweep_tasks == 0 && nf < sparse);
    const bool narrow_b = sweep_tasks == 2 || (sweep_tasks == 0 && nbk < sparse);
    if (narrow_f) sp.fwd_rt[l] = precision == 0 ? 16 : 64;
    if (narrow_b) sp.bwd_rows[l] = std::min(bwd_rows, precision == 0 ? 64 : 128);
    if (S.lev_ptr[l + 1] == S.lev_ptr[l]) continue;
    // the launchers pick the narrow kernels by shape (forward rows; chunk <= 128 / 64 rows)
    (narrow_f ? sp.fwd_narrow : sp.fwd_wide)++;
    (sp.bwd_rows[l] > (precision == 0 ? 64 : 128) ? sp.bwd_wide : sp.bwd_narrow)++;
    for (int32_t q = S.lev_ptr[l]; q < S.lev_ptr[l + 1]; q++) {
      const int s = S.lev_sn[q];
      const int k = S.sn_k[s], m = S.sn_m[s], r = m - k;
      if ((m + sp.bwd_rows[l] - 1) / sp.bwd_rows[l] > 1) sp.bwd_split += (k + 31) / 32;
      sp.max_k = std::max(sp.max_k, k);
      if (precision == 1 && r > 0) {
        const int64_t T = (r + 127) / 128;
        sp.tc_tiles += T * (T + 1) / 2;
        if (T > 1) sp.tc_multi++;
        sp.tc_kstages = std::max(sp.tc_kstages, (2 * k + 31) / 32);
      }
    }
  }
  return sp;
}

// (Re)builds the triangular-sweep task lists of F from its kept tree for the schedule sp:
// forward (supernode, row block) tasks, backward (supernode, column block, row chunk,
// finish record) tasks and their finish records, per-level offsets and shapes, the
// partial-sum buffer, and the variant counts.  Replaces any previous lists.
hz_status build_sweep_tasks(hz_ctx* c, hz::FactorDev& F, const SweepPlan& sp) {
  const int nlev = int(F.t_lev_ptr.size()) - 1;
  const int32_t *lev_ptr = F.t_lev_ptr.data(), *lev_sn = F.t_lev_sn.data();
  const int32_t *sn_k = F.t_sn_k.data(), *sn_m = F.t_sn_m.data();
  std::vector<int2> fwd;
  std::vector<int4> bwd, bfin;
  std::vector<int64_t> fwd_ptr(nlev + 1), bwd_ptr(nlev + 1), bfin_ptr(nlev + 1);
  int64_t max_bwd_level = 0;
  for (int l = 0; l < nlev; l++) {
    fwd_ptr[l] = int64_t(fwd.size());
    bwd_ptr[l] = int64_t(bwd.size());
    bfin_ptr[l] = int64_t(bfin.size());
    for (int32_t q = lev_ptr[l]; q < lev_ptr[l + 1]; q++) {
      const int s = lev_sn[q];
      const int k = sn_k[s], m = sn_m[s];
      const int frows = sp.fwd_rt[l];                  // forward task rows (k_fwd / k_fwd_c64)
      for (int rb = 0; rb * frows < m; rb++) fwd.push_back(make_int2(s, rb));
      const int nch = (m + sp.bwd_rows[l] - 1) / sp.bwd_rows[l];
      for (int cb = 0; cb * 32 < k; cb++) {
        const int fin = int(bfin.size());          // global index: its counter and its record
        bfin.push_back(make_int4(s, cb, int(int64_t(bwd.size()) - bwd_ptr[l]), nch));
        for (int ch = 0; ch < nch; ch++) bwd.push_back(make_int4(s, cb, ch, fin));
      }
    }
    max_bwd_level = std::max(max_bwd_level, int64_t(bwd.size()) - bwd_ptr[l]);
  }
  fwd_ptr[nlev] = int64_t(fwd.size());
  bwd_ptr[nlev] = int64_t(bwd.size());
  bfin_ptr[nlev] = int64_t(bfin.size());
  if (const char* vb = std::getenv("HZ_VERBOSE"); vb && std::atoi(vb) >= 2) {
    // per tree level: supernodes, panel entries and sweep tasks (for reading launch lists)
    for (int l = 0; l < nlev; l++) {
      int64_t pe = 0;
      for (int32_t q = lev_ptr[l]; q < lev_ptr[l + 1]; q++) {
        const int s = lev_sn[q];
        pe += int64_t(sn_k[s]) * (2 * sn_m[s] - sn_k[s] + 1) / 2;
      }
      std::fprintf(stderr, "[hz] level %3d: %6d supernodes %12lld panel entries %6lld fwd %6lld bwd tasks\n", l,
                   lev_ptr[l + 1] - lev_ptr[l], (long long)pe, (long long)(fwd_ptr[l + 1] - fwd_ptr[l]),
                   (long long)(bwd_ptr[l + 1] - bwd_ptr[l]));
    }
  }
  dfree(c, F.fwd_tasks);
  dfree(c, F.bwd_tasks);
  dfree(c, F.bfin_tasks);
  dfree(c, F.bwd_counters);
  dfree(c, F.bwd_partial);
  F.fwd_tasks = nullptr;
  F.bwd_tasks = nullptr;
  F.bfin_tasks = nullptr;
  F.bwd_counters = nullptr;
  F.bwd_partial = nullptr;
  TRY(upload(c, &F.fwd_tasks, fwd));
  TRY(upload(c, &F.bwd_tasks, bwd));
  TRY(upload(c, &F.bfin_tasks, bfin));
  TRY(upload(c, &F.bwd_counters, std::vector<unsigned int>(std::max<size_t>(bfin.size(), 1), 0u)));
  void* bp = nullptr;
  TRY(dalloc(c, (char**)&bp, std::max<int64_t>(max_bwd_level, 1) * 32 * int64_t(F.precision == 0 ? 16 : 8)));
  F.bwd_partial = bp;
  auto hcopy = [](const std::vector<int64_t>& v) {
    int64_t* p = new int64_t[v.size()];
    std::copy(v.begin(), v.end(), p);
    return p;
  };
  delete[] F.h_fwd_ptr;
  delete[] F.h_bwd_ptr;
  delete[] F.h_bfin_ptr;
  delete[] F.h_fwd_rt;
  delete[] F.h_bwd_rows;
  F.h_fwd_ptr = hcopy(fwd_ptr);
  F.h_bwd_ptr = hcopy(bwd_ptr);
  F.h_bfin_ptr = hcopy(bfin_ptr);
  F.h_fwd_rt = new int[nlev];
  F.h_bwd_rows = new int[nlev];
  std::copy(sp.fwd_rt.begin(), sp.fwd_rt.end(), F.h_fwd_rt);
  std::copy(sp.bwd_rows.begin(), sp.bwd_rows.end(), F.h_bwd_rows);
  F.v_fwd_wide = sp.fwd_wide;
  F.v_fwd_narrow = sp.fwd_narrow;
  F.v_bwd_wide = sp.bwd_wide;
  F.v_bwd_narrow = sp.bwd_narrow;
  F.v_bwd_split = sp.bwd_split;
  return HZ_OK;
}

// Sweep autotuner (hz_options.tune_sweeps): times the triangular sweeps of a factor
// (A_i^{-1} on every subdomain, or the coarse E^{-1}; forward and backward) under the
// schedules that scale the task count below which a level gets narrow tasks by 1/4, 1/2,
// 1 and 2 and cut wide backward
// chunks of 256 or 512 rows (complex64; 128 or 256 for complex128): one warm-up and three
// timed runs each, CUDA events on the context stream; the fastest is kept.  It runs at
// the first hz_factor, on the factor just computed and before any iteration graph holds
// the task lists.
hz_status tune_sweeps(hz_ctx* c, hz::FactorDev& F) {
  if (F.nsn == 0) return HZ_OK;
  const TreeView T{int(F.t_lev_ptr.size()) - 1, F.t_lev_ptr.data(), F.t_lev_sn.data(), F.t_sn_k.data(),
                   F.t_sn_m.data()};
  const int prec = F.precision;
  const int chunks[2] = {prec == 1 ? 256 : 128, prec == 1 ? 512 : 256};
  const double scales[4] = {0.25, 0.5, 1.0, 2.0};
  CU(cudaMemsetAsync(F.t_loc, 0, size_t(F.ntot) * (prec == 0 ? 16 : 8), c->st));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_chunk = chunks[1];
  double best_scale = 1.0;
  static const bool verbose = std::getenv("HZ_VERBOSE") != nullptr;
  for (int ch : chunks)
    for (double sc : scales) {
      TRY(build_sweep_tasks(c, F, plan_sweeps(T, prec, ch, 0, sc)));
      hz::launch_solve(F, c->st);
      CU(cudaEventRecord(e0, c->st));
      for (int r = 0; r < 3; r++) hz::launch_solve(F, c->st);
      CU(cudaEventRecord(e1, c->st));
      CU(cudaEventSynchronize(e1));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, e0, e1));
      if (verbose) std::fprintf(stderr, "[hz] sweep tuning: chunk %3d scale %.2f: %.3f ms\n", ch, sc, ms / 3);
      if (ms < best) {
        best = ms;
        best_chunk = ch;
        best_scale = sc;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TRY(build_sweep_tasks(c, F, plan_sweeps(T, prec, best_chunk, 0, best_scale)));
  F.sweep_chunk = best_chunk;
  F.sweep_scale = best_scale;
  return HZ_OK;
}

// sweep_tasks / bwd_chunk: hz_options fields of the same names (task shapes per level).
hz_status upload_factor(hz_ctx* c, const hz::SymbolicSet& S, int precision, int64_t nglob, hz::FactorDev& F,
                        double maxabs[3], int bwd_rows, int nrhs_block, int sweep_tasks, int bwd_chunk,
                        int merge_width = 0, int merge_sparse = 0) {
  F = hz::FactorDev();
  if (bwd_chunk > 0) bwd_rows = bwd_chunk;
  F.bwd_rows = bwd_rows;
  F.precision = precision;
  F.nmat = S.nmat;
  F.nsn = int(S.sn_k.size());
  F.nlev = S.nlev;
  F.ntot = S.voff.back();
  F.panel_elems = 0;   // set below from the padded layout
  F.u_elems = S.u_elems;
  F.front_elems = S.front_elems;
  F.nentries = int64_t(S.epos.size());
  F.nglob = nglob;
  const int ns = F.nsn;
  std::vector<hz::SnDev> sn(ns);
  int64_t panel_off = 0;
  for (int s = 0; s < ns; s++) {
    sn[s].k = S.sn_k[s];
    sn[s].m = S.sn_m[s];
    sn[s].first = S.sn_first[s];
    sn[s].parent = S.sn_parent[s];
    sn[s].rowoff = S.sn_rowoff[s];
    // complex64 panels: columns padded to 4 rows (32 bytes) for 16-byte vector loads
    sn[s].ld = precision == 0 ? S.sn_m[s] : (S.sn_m[s] + 3) / 4 * 4;
    sn[s].pad_ = 0;
    sn[s].paneloff = panel_off;
    panel_off += int64_t(sn[s].ld) * S.sn_k[s];
    sn[s].uoff = S.sn_uoff[s];
    sn[s].frontoff = S.sn_frontoff[s];
    F.maxk = std::max(F.maxk, S.sn_k[s]);
    F.maxm = std::max(F.maxm, S.sn_m[s]);
  }
  F.panel_elems = panel_off;
  const size_t vs = precision == 0 ? 16 : 8;
  TRY(upload(c, &F.sn, sn));
  // the solve tree: merged chains get their own panels after the factor's, filled at the end
  // of each factorisation (launch_merge_panels)
  const SolveTree ST = plan_solve_tree(S, merge_width, merge_sparse);
  {
    std::vector<hz::SnDev> ssn(ST.chains.size());
    int64_t off = panel_off;
    F.merges.clear();
    F.merge_tmp_elems = 0;
    for (size_t ci = 0; ci < ST.chains.size(); ci++) {
      const std::vector<int32_t>& ch = ST.chains[ci];
      if (ch.size() == 1) {
        ssn[ci] = sn[size_t(ch[0])];
        continue;
      }
      hz::SnDev& d = ssn[ci];
      d = sn[size_t(ch.front())];
      d.k = ST.k[ci];
      d.m = ST.m[ci];
      d.ld = precision == 0 ? d.m : (d.m + 3) / 4 * 4;     // complex64: 16-byte aligned row pairs
      d.parent = S.sn_parent[ch.back()];
      d.uoff = S.sn_uoff[ch.back()];
      d.paneloff = off;
      int w = 0;
      for (int32_t s : ch) {
        F.merges.push_back({off, sn[size_t(s)].paneloff, d.ld, w, sn[size_t(s)].ld, S.sn_k[s], S.sn_m[s]});
        F.merge_tmp_elems = std::max(F.merge_tmp_elems, int64_t(S.sn_k[s]) * w);
        w += S.sn_k[s];
      }
      off += int64_t(d.ld) * d.k;
    }
    F.solve_panel_elems = off;
    F.snlev = ST.nlev;
    TRY(upload(c, &F.ssn, ssn));
  }
  TRY(upload(c, &F.rowlist, S.rowlist));
  TRY(upload(c, &F.cptr, S.cptr));
  TRY(upload(c, &F.cidx, S.cidx));
  TRY(upload(c, &F.rel, S.rel));
  TRY(upload(c, &F.reloff, S.sn_reloff));
  TRY(upload(c, &F.gidx, S.gidx));
  TRY(upload(c, &F.epos, S.epos));
  TRY(upload(c, &F.ek, S.ek));
  TRY(upload(c, &F.em, to_d2(S.em)));
  TRY(upload(c, &F.eb, to_d2(S.eb)));
  for (size_t e = 0; e < S.ek.size(); e++) {
    maxabs[0] = std::max(maxabs[0], std::fabs(S.ek[e]));
    maxabs[1] = std::max(maxabs[1], std::abs(S.em[e]));
    maxabs[2] = std::max(maxabs[2], std::abs(S.eb[e]));
  }
  // gather-form prolongation (entries with zero weight are skipped)
  {
    std::vector<int64_t> pptr(nglob + 1, 0);
    for (int64_t q = 0; q < F.ntot; q++)
      if (S.weight[q] != 0.0) pptr[S.gidx[q] + 1]++;
    for (int64_t g = 0; g < nglob; g++) pptr[g + 1] += pptr[g];
    std::vector<int32_t> pidx(pptr[nglob]);
    std::vector<double> pw(pptr[nglob]);
    std::vector<int64_t> fill(pptr.begin(), pptr.end() - 1);
    for (int64_t q = 0; q < F.ntot; q++)
      if (S.weight[q] != 0.0) {
        const int64_t p = fill[S.gidx[q]]++;
        pidx[p] = int32_t(q);
        pw[p] = S.weight[q];
      }
    TRY(upload(c, &F.pptr, pptr));
    TRY(upload(c, &F.pidx, pidx));
    TRY(upload(c, &F.pw, pw));
  }
  // algorithmic bytes / flops of one forward + backward sweep
  {
    const double v = double(vs);
    double pan = 0, macs = 0, cb = 0, rows = 0;
    for (int s = 0; s < ns; s++) {
      const double k = S.sn_k[s], m = S.sn_m[s];
      pan += k * (k + 1) / 2 + (m - k) * k;
      macs += k * (k - 1) / 2 + (m - k) * k;
      cb += m - k;
      rows += m;
    }
    const double nt = double(F.ntot);
    const double fwd = pan * v + nt * v + cb * (v + 8) + rows * 8 + nt * v + cb * v;
    const double bwd = pan * v + nt * v + cb * (v + 4) + nt * v;
    F.solve_bytes = fwd + bwd;
    F.solve_flops = 8.0 * 2.0 * macs;
    F.gather_bytes = nt * (4 + 16 + v);
    int64_t pn = 0;
    for (int64_t q = 0; q < F.ntot; q++) pn += S.weight[q] != 0.0;
    F.prolong_nnz = pn;
    F.prolong_bytes = double(nglob + 1) * 8 + double(pn) * (4 + 8 + v) + double(nglob) * 16;
  }
  // task lists
  const int nlev = S.nlev;
  std::vector<int2> wg, ea;
  std::vector<int4> cbt, tct;
  std::vector<int64_t> scr_off(ns, 0);
  std::vector<std::vector<int32_t>> children(ns);
  for (int s = 0; s < ns; s++)
    if (S.sn_parent[s] >= 0) children[S.sn_parent[s]].push_back(s);
  int max_slot = 1;
  for (int s = 0; s < ns; s++) max_slot = std::max(max_slot, int(children[s].size()));
  F.max_slot = max_slot;
  std::vector<int64_t> lev_ptr(nlev + 1), wg_ptr(nlev + 1), cb_ptr(nlev + 1), ea_ptr(int64_t(nlev) * max_slot + 1),
      tc_ptr(nlev + 1);
  int64_t scratch = 0;
  // factorisation groups: per level (and extend-add slot) the start of each group's
  // tasks; every list is ordered by supernode within a level, hence by group
  const int G = std::max(1, int(S.grp_sn.size()) - 1);
  const std::vector<int32_t> grp_sn = S.grp_sn.size() >= 2 ? S.grp_sn : std::vector<int32_t>{0, ns};
  auto grp_of = [&](int sn) { return int(std::upper_bound(grp_sn.begin(), grp_sn.end(), sn) - grp_sn.begin()) - 1; };
  std::vector<int64_t> lev_g(size_t(nlev) * (G + 1)), wg_g(lev_g.size()), cb_g(lev_g.size()), tc_g(lev_g.size()),
      ea_g(size_t(nlev) * max_slot * (G + 1));
  struct Split {                      // fills out[base + g] with the list size where group g starts
    std::vector<int64_t>& out;
    size_t base;
    int G, next;
    void enter(int g, int64_t size) { while (next <= g) out[base + next++] = size; }
    void finish(int64_t size) { while (next <= G) out[base + next++] = size; }
  };
  const SweepPlan sp = plan_sweeps(ST.view(), precision, bwd_rows, sweep_tasks);
  const SweepPlan spf = plan_sweeps(view_of(S), precision, bwd_rows, sweep_tasks);   // factor-side counts
  F.v_fwd_wide = sp.fwd_wide;
  F.v_fwd_narrow = sp.fwd_narrow;
  F.v_bwd_wide = sp.bwd_wide;
  F.v_bwd_narrow = sp.bwd_narrow;
  F.v_bwd_split = sp.bwd_split;
  F.v_tc_tiles = spf.tc_tiles;
  F.v_tc_multi = spf.tc_multi;
  F.v_tc_kstages = spf.tc_kstages;
  F.v_max_k = spf.max_k;
  for (int l = 0; l < nlev; l++) {
    lev_ptr[l] = S.lev_ptr[l];
    wg_ptr[l] = int64_t(wg.size());
    cb_ptr[l] = int64_t(cbt.size());
    tc_ptr[l] = int64_t(tct.size());
    int64_t lev_scr = 0;
    int cur_g = -1;
    Split sl{lev_g, size_t(l) * (G + 1), G, 0}, sw{wg_g, size_t(l) * (G + 1), G, 0},
        sc{cb_g, size_t(l) * (G + 1), G, 0}, st{tc_g, size_t(l) * (G + 1), G, 0};
    for (int32_t q = S.lev_ptr[l]; q < S.lev_ptr[l + 1]; q++) {
      const int s = S.lev_sn[q];
      const int k = S.sn_k[s], m = S.sn_m[s], r = m - k;
      const int gs = grp_of(s);
      if (gs != cur_g) {                           // a group's W blocks start the scratch again
        cur_g = gs;
        lev_scr = 0;
        sl.enter(gs, q);
        sw.enter(gs, int64_t(wg.size()));
        sc.enter(gs, int64_t(cbt.size()));
        st.enter(gs, int64_t(tct.size()));
      }
      for (int rb = 0; rb * 32 < r; rb++) wg.push_back(make_int2(s, rb));
      if (precision == 0) {
        const int T = (r + 31) / 32;
        for (int ti = 0; ti < T; ti++)
          for (int tj = 0; tj <= ti; tj++) cbt.push_back(make_int4(s, ti, tj, 0));
      } else {
        const int T = (r + 127) / 128;
        for (int ti = 0; ti < T; ti++)
          for (int tj = 0; tj <= ti; tj++) tct.push_back(make_int4(s, ti, tj, 0));
      }
      scr_off[s] = lev_scr;
      lev_scr += int64_t(r) * k;
      scratch = std::max(scratch, lev_scr);
    }
    sl.finish(S.lev_ptr[l + 1]);
    sw.finish(int64_t(wg.size()));
    sc.finish(int64_t(cbt.size()));
    st.finish(int64_t(tct.size()));
    for (int q = 0; q < max_slot; q++) {
      ea_ptr[int64_t(l) * max_slot + q] = int64_t(ea.size());
      Split se{ea_g, (size_t(l) * max_slot + q) * (G + 1), G, 0};
      for (int32_t z = S.lev_ptr[l]; z < S.lev_ptr[l + 1]; z++) {
        const int p = S.lev_sn[z];
        se.enter(grp_of(p), int64_t(ea.size()));
        if (q < int(children[p].size())) {
          const int ch = children[p][q];
          const int r = S.sn_m[ch] - S.sn_k[ch];
          for (int cb = 0; cb * 8 < r; cb++) ea.push_back(make_int2(ch, cb));
        }
      }
      se.finish(int64_t(ea.size()));
    }
  }
  lev_ptr[nlev] = S.lev_ptr[nlev];
  wg_ptr[nlev] = int64_t(wg.size());
  cb_ptr[nlev] = int64_t(cbt.size());
  tc_ptr[nlev] = int64_t(tct.size());
  ea_ptr[int64_t(nlev) * max_slot] = int64_t(ea.size());
  F.scratch_elems = scratch;
  TRY(upload(c, &F.wg_tasks, wg));
  TRY(upload(c, &F.cb_tasks, cbt));
  TRY(upload(c, &F.tc_tasks, tct));
  TRY(upload(c, &F.ea_tasks, ea));
  TRY(upload(c, &F.scr_off, scr_off));
  TRY(upload(c, &F.lev_sn, S.lev_sn));
  auto hcopy = [](const std::vector<int64_t>& v) {
    int64_t* p = new int64_t[v.size()];
    std::copy(v.begin(), v.end(), p);
    return p;
  };
  F.h_lev_ptr = hcopy(lev_ptr);
  F.h_wg_ptr = hcopy(wg_ptr);
  F.h_cb_ptr = hcopy(cb_ptr);
  F.h_tc_ptr = hcopy(tc_ptr);
  F.h_ea_ptr = hcopy(ea_ptr);
  F.h_ent_ptr = hcopy(S.ent_ptr);
  F.ngrp = G;
  F.h_lev_g = hcopy(lev_g);
  F.h_wg_g = hcopy(wg_g);
  F.h_cb_g = hcopy(cb_g);
  F.h_tc_g = hcopy(tc_g);
  F.h_ea_g = hcopy(ea_g);
  F.h_ent_g = hcopy(S.ent_gptr.size() == size_t(nlev) * (G + 1) ? S.ent_gptr : [&] {
    std::vector<int64_t> v(size_t(nlev) * (G + 1));      // one group: the level's whole range
    for (int l = 0; l < nlev; l++) {
      v[size_t(l) * (G + 1)] = S.ent_ptr[l];
      v[size_t(l) * (G + 1) + 1] = S.ent_ptr[l + 1];
    }
    return v;
  }());
  // the (solve) tree as the sweep schedule sees it, kept for the sweep autotuner
  F.t_lev_ptr = ST.lev_ptr;
  F.t_lev_sn = ST.lev_sn;
  F.t_sn_k = ST.k;
  F.t_sn_m = ST.m;
  TRY(build_sweep_tasks(c, F, sp));
  F.sweep_chunk = bwd_rows;
  F.sweep_scale = 1.0;
  // batched sweeps for nrhs_block right-hand sides (pseudo-block FGMRES)
  if (nrhs_block > 1) {
    F.mS = nrhs_block;
    F.mbwd_rows = 128;
    std::vector<int2> mf;
    std::vector<int4> mb, mfin;
    std::vector<int64_t> mf_ptr(nlev + 1), mb_ptr(nlev + 1);
    int64_t max_mb = 0;
    for (int l = 0; l < nlev; l++) {
      mf_ptr[l] = int64_t(mf.size());
      mb_ptr[l] = int64_t(mb.size());
      for (int32_t q = S.lev_ptr[l]; q < S.lev_ptr[l + 1]; q++) {
        const int s = S.lev_sn[q];
        const int k = S.sn_k[s], m = S.sn_m[s];
        for (int rb = 0; rb * 64 < m; rb++) mf.push_back(make_int2(s, rb));
        const int nch = (m + F.mbwd_rows - 1) / F.mbwd_rows;
        for (int cb = 0; cb * 32 < k; cb++) {
          const int fin = int(mfin.size());
          mfin.push_back(make_int4(s, cb, int(int64_t(mb.size()) - mb_ptr[l]), nch));
          for (int ch = 0; ch < nch; ch++) mb.push_back(make_int4(s, cb, ch, fin));
        }
      }
      max_mb = std::max(max_mb, int64_t(mb.size()) - mb_ptr[l]);
    }
    mf_ptr[nlev] = int64_t(mf.size());
    mb_ptr[nlev] = int64_t(mb.size());
    TRY(upload(c, &F.mfwd_tasks, mf));
    TRY(upload(c, &F.mbwd_tasks, mb));
    TRY(upload(c, &F.mbfin_tasks, mfin));
    TRY(upload(c, &F.mbwd_counters, std::vector<unsigned int>(std::max<size_t>(mfin.size(), 1), 0u)));
    F.h_mfwd_ptr = new int64_t[nlev + 1];
    F.h_mbwd_ptr = new int64_t[nlev + 1];
    std::copy(mf_ptr.begin(), mf_ptr.end(), F.h_mfwd_ptr);
    std::copy(mb_ptr.begin(), mb_ptr.end(), F.h_mbwd_ptr);
    const int64_t vsz = int64_t(vs) * nrhs_block;
    void *a = nullptr, *b = nullptr, *d = nullptr, *e = nullptr, *f = nullptr;
    TRY(dalloc(c, (char**)&a, F.ntot * vsz));
    TRY(dalloc(c, (char**)&b, F.ntot * vsz));
    TRY(dalloc(c, (char**)&d, F.ntot * vsz));
    TRY(dalloc(c, (char**)&e, std::max<int64_t>(F.u_elems, 1) * vsz));
    TRY(dalloc(c, (char**)&f, std::max<int64_t>(max_mb, 1) * 32 * vsz));
    F.mt_loc = a;
    F.mz_loc = b;
    F.mx_loc = d;
    F.mu_ws = e;
    F.mbwd_partial = f;
  }
  // numeric storage and solve workspaces
  void *pan = nullptr, *tl = nullptr, *zl = nullptr, *xl = nullptr, *uw = nullptr;
  TRY(dalloc(c, (char**)&pan, F.solve_panel_elems * int64_t(vs)));
  if (F.merge_tmp_elems > 0) TRY(dalloc(c, (char**)&F.merge_tmp, F.merge_tmp_elems * int64_t(vs)));
  TRY(dalloc(c, (char**)&tl, F.ntot * int64_t(vs)));
  TRY(dalloc(c, (char**)&zl, F.ntot * int64_t(vs)));
  TRY(dalloc(c, (char**)&xl, F.ntot * int64_t(vs)));
  TRY(dalloc(c, (char**)&uw, std::max<int64_t>(F.u_elems, 1) * int64_t(vs)));
  F.panels = pan;
  F.t_loc = tl;
  F.z_loc = zl;
  F.x_loc = xl;
  F.u_ws = uw;
  return HZ_OK;
}

void free_host_ptrs(hz::FactorDev& F) {
  delete[] F.h_lev_ptr;
  delete[] F.h_fwd_ptr;
  delete[] F.h_bwd_ptr;
  delete[] F.h_bfin_ptr;
  delete[] F.h_wg_ptr;
  delete[] F.h_cb_ptr;
  delete[] F.h_tc_ptr;
  F.h_tc_ptr = nullptr;
  delete[] F.h_ea_ptr;
  delete[] F.h_ent_ptr;
  delete[] F.h_lev_g;
  delete[] F.h_ent_g;
  delete[] F.h_wg_g;
  delete[] F.h_cb_g;
  delete[] F.h_tc_g;
  delete[] F.h_ea_g;
  F.h_lev_g = F.h_ent_g = F.h_wg_g = F.h_cb_g = F.h_tc_g = F.h_ea_g = nullptr;
  delete[] F.h_mfwd_ptr;
  delete[] F.h_fwd_rt;
  delete[] F.h_bwd_rows;
  F.h_fwd_rt = nullptr;
  F.h_bwd_rows = nullptr;
  delete[] F.h_mbwd_ptr;
  F.h_mfwd_ptr = F.h_mbwd_ptr = nullptr;
  F.h_bfin_ptr = F.h_lev_ptr = F.h_fwd_ptr = F.h_bwd_ptr = F.h_wg_ptr = F.h_cb_ptr = F.h_ea_ptr = F.h_ent_ptr = nullptr;
}

hz_status factor_one(hz_ctx* c, hz::FactorDev& F, double w, const double maxabs[3], double& min_pivot) {
  if (F.nsn == 0) return HZ_OK;
  static const bool verbose = std::getenv("HZ_VERBOSE") != nullptr;
  auto t0 = std::chrono::steady_clock::now();
  const size_t vs = F.precision == 0 ? 16 : 8;
  char *fronts = nullptr, *scratch = nullptr;
  TRY(dalloc(c, &fronts, F.front_elems * int64_t(vs)));
  hz_status s = dalloc(c, &scratch, std::max<int64_t>(F.scratch_elems, 1) * int64_t(vs));
  if (s != HZ_OK) {
    dfree(c, fronts);
    return s;
  }
  hz::DevStatus init{0u, 0u, 0.0};   // zero_pivot, timeout, min_pivot
  const double big = 1e300;
  std::memcpy(&init.min_pivot, &big, sizeof(double));
  CU(cudaMemcpyAsync(c->status, &init, sizeof(init), cudaMemcpyHostToDevice, c->st));
  const double tiny = 1e-13 * (maxabs[0] + w * w * maxabs[1] + w * maxabs[2]);
  if (verbose) {
    cudaStreamSynchronize(c->st);
    std::fprintf(stderr, "[hz] factor: workspace %.2f GB allocated in %.3f s\n",
                 double(F.front_elems) * double(vs) / 1e9,
                 std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    t0 = std::chrono::steady_clock::now();
  }
  for (int g = 0; g < F.ngrp; g++)                 // groups one after the other in one workspace
    for (int l = 0; l < F.nlev; l++) hz::launch_factor_level(F, l, g, w, fronts, scratch, c->status, tiny, c->st);
  hz::launch_merge_panels(F, c->st);              // merged solve supernodes of the sweeps
  if (verbose) {
    cudaStreamSynchronize(c->st);
    std::fprintf(stderr, "[hz] factor: %d levels in %.3f s\n", F.nlev,
                 std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    t0 = std::chrono::steady_clock::now();
  }
  CU(cudaGetLastError());
  hz::DevStatus out{};
  CU(cudaMemcpyAsync(&out, c->status, sizeof(out), cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  dfree(c, fronts);
  dfree(c, scratch);
  if (verbose)
    std::fprintf(stderr, "[hz] factor: status read and workspace freed in %.3f s\n",
                 std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  min_pivot = std::min(min_pivot, out.min_pivot);
  if (out.timeout)
    return fail(c, HZ_ERR_TIMEOUT, (out.timeout & 2u)
                                       ? "a tensor-core completion wait and its drain wait ran out in the factorisation"
                                       : "a tensor-core completion wait ran out in the factorisation");
  if (out.zero_pivot) return fail(c, HZ_ERR_ZERO_PIVOT, "tiny pivot in a local LDL^T factor");
  return HZ_OK;
}

// y ~ E^{-1} r (iterative coarse solve): one cycle of GMRES(coarse_maxit) on E
// right-preconditioned by one-level ORAS on the coarse mesh (Eq. 4 with the coarse
// subdomains), CGS2 and the Givens rotations of the outer solve, x0 = 0, ending when
// the estimate |g_{j+1}| / ||r|| reaches coarse_tol, on a happy breakdown or after
// coarse_maxit iterations.  Host-synchronous: one pinned read per inner iteration.
// r is not modified; a zero r gives y = 0.
void coarse_inner(hz_ctx* c, const double2* r, double2* y) {
  const int64_t nH = c->nH;
  const int mH = c->cmaxit;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  double* pin = c->h_pin + hz_ctx::PIN_CRS;
  hz::launch_cgs(nH, 0, c->VH, nH, nullptr, const_cast<double2*>(r), 0, c->partial, st);
  hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
  cudaMemsetAsync(y, 0, size_t(nH) * 16, st);
  cudaMemcpyAsync(pin, &c->nrm[64].x, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (!(pin[0] > 0.0) || !std::isfinite(pin[0])) {
    c->stats.coarse_solves++;
    return;
  }
  hz::launch_init_cycle(c->nrm, c->gH, mH, c->scalH + 2, c->scalH + 3, st);
  hz::launch_scale(nH, r, c->scalH + 2, c->VH, st);
  int k = 0;
  for (int j = 0; j < mH; j++) {
    double2* vj = c->VH + int64_t(j) * nH;
    double2* zj = c->ZH + int64_t(j) * nH;
    hz::launch_gather(c->cloc, vj, st);                                           // R_H,i v
    hz::launch_solve(c->cloc, st);                                                // E_i^{-1}
    hz::launch_prolong(c->cloc, nullptr, zj, st);                                 // sum R^T D x_i
    hz::launch_spmv(nH, c->d_Erp, c->d_Eci, c->d_E, zj, nullptr, c->wH, st);      // E z_j
    hz::launch_cgs(nH, j + 1, c->VH, nH, nullptr, c->wH, j + 1, c->partial, st);
    hz::launch_reduce(c->partial, nb, j + 1, c->h1, st);
    hz::launch_cgs(nH, j + 1, c->VH, nH, c->h1, c->wH, j + 1, c->partial, st);
    hz::launch_reduce(c->partial, nb, j + 1, c->h2, st);
    hz::launch_cgs(nH, j + 1, c->VH, nH, c->h2, c->wH, 0, c->partial, st);
    hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
    hz::launch_givens(j, mH, c->HH, c->csH, c->snH, c->gH, c->h1, c->h2, c->nrm, c->scalH + 3, c->scalH, c->brkH,
                      c->scalH + 1, st);
    hz::launch_scale(nH, c->wH, c->scalH + 1, c->VH + int64_t(j + 1) * nH, st);
    cudaMemcpyAsync(pin + 1, c->scalH, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(pin + 2, c->brkH, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    k = j + 1;
    int brk = 0;
    std::memcpy(&brk, pin + 2, sizeof(int));
    if (brk || !(pin[1] > c->ctol)) break;
  }
  hz::launch_update_x(nH, k, c->HH, mH + 1, c->gH, c->yHs, c->ZH, nH, y, st);
  c->stats.coarse_solves++;
  c->stats.coarse_iterations += k;
}

// y_H = E^{-1} r_H on the coarse factor (direct) or by the inner GMRES (iterative).
void coarse_solve(hz_ctx* c, const double2* r, double2* y) {
  if (c->coarse_oras) {
    coarse_inner(c, r, y);
    return;
  }
  hz::launch_gather(c->crs, r, c->st);
  hz::launch_solve(c->crs, c->st);
  hz::launch_prolong(c->crs, nullptr, y, c->st);
}

// z = M^{-1} v  (Eq. 3 with two levels, Eq. 4 with one)
void apply_prec(hz_ctx* c, const double2* v, double2* z) {
  cudaStream_t st = c->st;
  if (c->levels == 2) {
    hz::launch_spmv_real(c->nH, c->d_Ztrp, c->d_Ztci, c->d_Ztv, v, c->rH, st);   // r_H = Z^T v
    coarse_solve(c, c->rH, c->yH);                                               // E^{-1}
    hz::launch_spmv_real(c->n, c->d_Zrp, c->d_Zci, c->d_Zv, c->yH, c->y, st);     // y = Z y_H
    hz::launch_spmv(c->n, c->d_rp, c->d_ci, c->d_A, c->y, v, c->t, st);          // t = v - A y
    hz::launch_gather(c->loc, c->t, st);                                         // R_i t
    hz::launch_solve(c->loc, st);                                                // A_i^{-1}
    hz::launch_prolong(c->loc, c->y, z, st);                                     // y + sum R_i^T D_i x_i
  } else {
    hz::launch_gather(c->loc, v, st);
    hz::launch_solve(c->loc, st);
    hz::launch_prolong(c->loc, nullptr, z, st);
  }
}


hz_status norm2(hz_ctx* c, const double2* v, double& out) {
  const int nb = hz::cgs_blocks();
  hz::launch_cgs(c->n, 0, c->V, c->n, nullptr, const_cast<double2*>(v), 0, c->partial, c->st);
  hz::launch_reduce(c->partial, nb, 0, c->nrm, c->st);
  CU(cudaMemcpyAsync(c->h_pin + 5, &c->nrm[64].x, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  out = std::sqrt(c->h_pin[5]);
  return HZ_OK;
}

// Kernels of inner iteration j: z_j = M^{-1} v_j, w = A z_j, CGS2 against v_0..v_j,
// Givens update, v_{j+1} = w / h_{j+1,j}, and the copy of the residual estimate and
// breakdown flag to pinned host memory.  The same sequence serves eager launches
// and the capture of iteration j's CUDA graph.
void iteration_kernels(hz_ctx* c, int j) {
  const int64_t n = c->n;
  const int m = c->restart;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  double2* vj = c->V + int64_t(j) * n;
  double2* zj = c->Zs + int64_t(j) * n;
  apply_prec(c, vj, zj);
  hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, zj, nullptr, c->w, st);
  // orthogonalise against [C, v_0..v_j] (C: the recycled space, empty without recycling)
  const int kk = c->ckk, nc = kk + j + 1;
  const double2* base = c->V - int64_t(kk) * n;
  hz::launch_cgs(n, nc, base, n, nullptr, c->w, nc, c->partial, st);        // h1, |w|
  hz::launch_reduce(c->partial, nb, nc, c->h1, st);
  hz::launch_cgs(n, nc, base, n, c->h1, c->w, nc, c->partial, st);          // w -= [C V] h1; h2
  hz::launch_reduce(c->partial, nb, nc, c->h2, st);
  hz::launch_cgs(n, nc, base, n, c->h2, c->w, 0, c->partial, st);           // w -= [C V] h2; |w|
  hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
  hz::launch_givens(j, m, c->H, c->cs, c->sn, c->g, c->h1, c->h2, c->nrm, c->scal + 4, c->scal, c->brk,
                    c->scal + 1, st, kk, c->rk ? c->Hraw : nullptr, c->Braw, c->rk);
  hz::launch_scale(n, c->w, c->scal + 1, c->V + int64_t(j + 1) * n, st);
  cudaMemcpyAsync(c->h_pin, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(c->h_pin + 4, c->brk, sizeof(int), cudaMemcpyDeviceToHost, st);
}

// Runs iteration j (as a CUDA graph when the stream can be captured) and waits for it.
hz_status run_iteration(hz_ctx* c, int j) {
  cudaStream_t st = c->st;
  const size_t gi = size_t(j) + size_t(c->restart) * size_t(c->ckk);
  if (c->graphs && st != nullptr) {
    if (!c->gexec[gi]) {
      const long long l0 = hz::launch_count();
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        iteration_kernels(c, j);
        if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) {
          if (cudaGraphInstantiate(&c->gexec[gi], g, 0) != cudaSuccess) c->gexec[gi] = nullptr;
          cudaGraphDestroy(g);
        }
      }
      cudaGetLastError();
      c->gcount[gi] = hz::launch_count() - l0;
      hz::add_launches(-c->gcount[gi]);          // capture itself launches nothing
      if (!c->gexec[gi]) c->graphs = false;     // this stream cannot be captured: stay eager
    }
    if (c->gexec[gi]) {
      CU(cudaGraphLaunch(c->gexec[gi], st));
      hz::add_launches(c->gcount[gi]);
      CU(cudaStreamSynchronize(st));
      return HZ_OK;
    }
  }
  iteration_kernels(c, j);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return HZ_OK;
}

// One right-hand side: FGMRES(m), CGS2, complex Givens (x0 = 0).
hz_status fgmres_one(hz_ctx* c, double tol, hz_rhs_info* info) {
  const int64_t n = c->n;
  const int m = c->restart;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  double bnorm = 0;
  TRY(norm2(c, c->b, bnorm));
  CU(cudaMemsetAsync(c->x, 0, size_t(n) * 16, st));
  info->iterations = 0;
  info->status = HZ_OK;
  info->rel_residual = 0.0;
  if (bnorm == 0.0) return HZ_OK;
  if (!std::isfinite(bnorm)) {
    info->status = HZ_ERR_BREAKDOWN;
    return HZ_OK;
  }
  double* d_invbeta = c->scal + 2;
  double* d_beta = c->scal + 3;
  c->h_pin[6] = bnorm;
  CU(cudaMemcpyAsync(c->scal + 4, c->h_pin + 6, sizeof(double), cudaMemcpyHostToDevice, st));
  // r = b
  hz::launch_axpby_copy(n, c->b, c->w, st);
  hz::launch_cgs(n, 0, c->V, n, nullptr, c->w, 0, c->partial, st);
  hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
  int its = 0;
  for (;;) {
    hz::launch_init_cycle(c->nrm, c->g, m, d_invbeta, d_beta, st);
    hz::launch_scale(n, c->w, d_invbeta, c->V, st);
    int k = 0;
    bool stop_nonfinite = false;
    for (int j = 0; j < m; j++) {
      TRY(run_iteration(c, j));
      its++;
      k = j + 1;
      const double est = c->h_pin[0];
      int brk = 0;
      std::memcpy(&brk, c->h_pin + 4, sizeof(int));
      if (!std::isfinite(est)) { stop_nonfinite = true; break; }
      if (brk || est <= tol || its >= c->max_iter) break;
    }
    if (stop_nonfinite) {
      info->iterations = its;
      info->status = HZ_ERR_BREAKDOWN;
      info->rel_residual = NAN;
      return HZ_OK;
    }
    hz::launch_update_x(n, k, c->H, m + 1, c->g, c->ysol, c->Zs, n, c->x, st);
    hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, c->x, c->b, c->w, st);        // r = b - A x
    double rn = 0;
    TRY(norm2(c, c->w, rn));
    const double rel = rn / bnorm;
    info->iterations = its;
    info->rel_residual = rel;
    if (!std::isfinite(rel)) {
      info->status = HZ_ERR_BREAKDOWN;
      return HZ_OK;
    }
    if (rel <= tol) return HZ_OK;
    if (its >= c->max_iter) {
      info->status = HZ_ERR_NOT_CONVERGED;
      return HZ_OK;
    }
    // nrm still holds |r|^2 from norm2 for the next cycle
  }
}

// ---------------------------------------------------------------------------
// GCRO-DR (options.recycle = rk > 0): FGMRES with deflated restarting and a recycled
// Krylov space kept across right-hand sides (Parks et al. 2006; the Krylov-recycling
// step the paper names for many right-hand sides).  Right preconditioning: the space
// lives in the preconditioned space (Uh) and in the solution space (Ux = M^{-1} Uh),
// with C = A Ux, C^H C = I.  Each cycle orthogonalises against [C, V]; the recycled
// space is renewed at every cycle end from harmonic Ritz vectors, on the host for the
// small matrices (order <= restart + 1) and on the device for the n-vectors.
// ---------------------------------------------------------------------------
using hz_small::cplx;

std::vector<cplx> to_host(const double2* d, size_t count) {
  std::vector<cplx> h(count);
  cudaMemcpy(h.data(), d, count * 16, cudaMemcpyDeviceToHost);
  return h;
}

// out (+)= sign * ([B1, B2] coef) with a host coefficient matrix.
void combo(hz_ctx* c, int nb1, const double2* B1, int nb2, const double2* B2, const std::vector<cplx>& coef,
           int nout, double2* out, double sign, bool acc) {
  cudaMemcpyAsync(c->dcoef, coef.data(), coef.size() * 16, cudaMemcpyHostToDevice, c->st);
  hz::launch_combo(c->n, nb1, B1, c->n, nb2, B2, c->n, c->dcoef, nout, out, c->n, sign, acc, c->st);
  cudaStreamSynchronize(c->st);                      // coef is a host temporary
}

// Indices of the kn eigenvalues of smallest modulus (stable order).
std::vector<int> smallest(const std::vector<cplx>& w, int kn) {
  std::vector<int> idx(w.size());
  for (size_t i = 0; i < w.size(); i++) idx[i] = int(i);
  auto key = [&](int a) {
    const double f = std::abs(w[size_t(a)]);
    return std::isfinite(f) ? f : 1e300;
  };
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return key(a) < key(b); });
  idx.resize(size_t(kn));
  return idx;
}

// out (+)= sign * [B_1, B_2, ...] coef for any number of columns (coef: total columns x
// nout, column-major, host).  The columns go to the combination kernel in pieces of at
// most kComboMaxCols; the first piece writes out (or adds to it, acc), the others add.
hz_status combo_cols(hz_ctx* c, const std::vector<std::pair<const double2*, int>>& blocks,
                     const std::vector<cplx>& coef, int nout, double2* out, double sign, bool acc) {
  int total = 0;
  for (const auto& b : blocks) total += b.second;
  bool first = true;
  int col = 0;
  for (const auto& b : blocks) {
    for (int a = 0; a < b.second; a += hz::kComboMaxCols) {
      const int w = std::min(hz::kComboMaxCols, b.second - a);
      std::vector<cplx> piece(size_t(w) * nout);
      for (int q = 0; q < nout; q++)
        for (int i = 0; i < w; i++) piece[size_t(q) * w + i] = coef[size_t(q) * total + col + a + i];
      combo(c, w, b.first + int64_t(a) * c->n, 0, nullptr, piece, nout, out, sign, acc || !first);
      first = false;
    }
    col += b.second;
  }
  if (first && !acc) CU(cudaMemsetAsync(out, 0, size_t(nout) * c->n * 16, c->st));
  CU(cudaGetLastError());
  return HZ_OK;
}

// The basis whose columns the recycled space C precedes in memory: C sits in the kk
// columns right before it, so that [C, V] is one column-major block.
double2* recycle_basis(hz_ctx* c) { return c->krylov == HZ_KRYLOV_BLOCK ? c->Vb : c->V; }

// New recycled space from the cycle that just ended, for one right-hand side (s = 1) or a
// block of s: kk recycled vectors at the cycle start, kc basis columns in the cycle (Arnoldi
// steps times s).  Hm ((kc + s) x kc) is the unrotated (block) Hessenberg matrix and Bm
// (kk x kc) the coefficients of the orthogonalisation against C, both column-major on the
// host; V (with C before it) and Z are the cycle's bases.  The k harmonic Ritz vectors of
// smallest |theta| over the search space become the new space:
//   kk = 0:  (H + H^{-H} E (H_+^H H_+) E^H) z = theta z, H the square top of Hm, H_+ the
//            s x s block below it, E the last s columns of the identity;
//   kk > 0:  G^H G z = theta G^H (Vh^H Wh) z, G = [[D, B], [0, Hm]], Vh = [C, V],
//            Wh = [Uh D, V_kc], D = diag(1 / |Uh_i|).
// With P the chosen vectors and G P = Q R: C = Vh Q, Uh = Wh P R^{-1}, Ux = [Ux D, Z] P R^{-1}
// (Parks et al. 2006, GCRO-DR; the block form replaces h_{m+1,m} by H_+).  On a numerical
// failure the previous space is kept.
hz_status recycle_space(hz_ctx* c, int kk, int kc, int s, const std::vector<cplx>& Hm, const std::vector<cplx>& Bm,
                        double2* V, const double2* Z) {
  const int rk = c->rk;
  const int64_t n = c->n;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  if (kc < 1) return HZ_OK;
  CU(cudaStreamSynchronize(st));
  const int lh = kc + s;                                                 // rows of Hm
  auto H = [&](int i, int j) { return Hm[size_t(j) * lh + i]; };
  const int nt = kk + kc;                                                // columns of G
  const int ng = nt + s;                                                 // rows of G
  const int kn = std::min(rk, nt);
  std::vector<cplx> G(size_t(ng) * nt, 0.0), P, w, VR, Mg;
  std::vector<double> dsc(size_t(kk), 1.0);
  std::string err;
  double2* Cb = V - int64_t(kk) * n;
  if (kk == 0) {
    std::vector<cplx> Hq(size_t(kc) * kc), HqH(size_t(kc) * kc), F(size_t(kc) * s, 0.0), HpHp(size_t(s) * s, 0.0);
    for (int j = 0; j < kc; j++)
      for (int i = 0; i < kc; i++) Hq[size_t(j) * kc + i] = H(i, j);
    for (int j = 0; j < kc; j++)
      for (int i = 0; i < kc; i++) HqH[size_t(j) * kc + i] = std::conj(Hq[size_t(i) * kc + j]);
    for (int q = 0; q < s; q++) F[size_t(q) * kc + kc - s + q] = 1.0;              // E
    if (!hz_small::lu_solve(kc, HqH, F, s)) return HZ_OK;                         // H^{-H} E
    for (int a = 0; a < s; a++)                                                    // H_+^H H_+
      for (int b = 0; b < s; b++) {
        cplx acc = 0;
        for (int r = 0; r < s; r++) acc += std::conj(H(kc + r, kc - s + a)) * H(kc + r, kc - s + b);
        HpHp[size_t(b) * s + a] = acc;
      }
    Mg = Hq;
    for (int b = 0; b < s; b++)
      for (int i = 0; i < kc; i++) {
        cplx acc = 0;
        for (int a = 0; a < s; a++) acc += F[size_t(a) * kc + i] * HpHp[size_t(b) * s + a];
        Mg[size_t(kc - s + b) * kc + i] += acc;
      }
    for (int j = 0; j < kc; j++)
      for (int i = 0; i < lh; i++) G[size_t(j) * ng + i] = H(i, j);
  } else {
    // Vh^H Wh = [[C^H Uh D, 0], [V^H Uh D, I_kc; 0]]: the Uh columns against [C, V], 64 at a time
    std::vector<cplx> VW(size_t(ng) * nt, 0.0);
    for (int i = 0; i < kk; i++) {
      double2* ui = c->Uh + int64_t(i) * n;
      double unorm2 = 0.0;
      for (int a = 0; a < ng; a += 64) {
        const int wc = std::min(64, ng - a);
        hz::launch_cgs(n, wc, Cb + int64_t(a) * n, n, nullptr, ui, wc, c->partial, st);
        hz::launch_reduce(c->partial, nb, wc, c->h1, st);
        CU(cudaStreamSynchronize(st));
        const std::vector<cplx> hv = to_host(c->h1, 65);
        for (int q = 0; q < wc; q++) VW[size_t(i) * ng + a + q] = hv[size_t(q)];
        unorm2 = hv[64].real();
      }
      dsc[size_t(i)] = 1.0 / std::sqrt(unorm2);
      for (int a = 0; a < ng; a++) VW[size_t(i) * ng + a] *= dsc[size_t(i)];
    }
    for (int j = 0; j < kc; j++) VW[size_t(kk + j) * ng + kk + j] = 1.0;
    for (int i = 0; i < kk; i++) G[size_t(i) * ng + i] = dsc[size_t(i)];
    for (int j = 0; j < kc; j++) {
      for (int i = 0; i < kk; i++) G[size_t(kk + j) * ng + i] = Bm[size_t(j) * kk + i];
      for (int i = 0; i < lh; i++) G[size_t(kk + j) * ng + kk + i] = H(i, j);
    }
    std::vector<cplx> Ag(size_t(nt) * nt, 0.0), Bg(size_t(nt) * nt, 0.0);
    for (int a = 0; a < nt; a++)
      for (int b = 0; b < nt; b++) {
        cplx sa = 0, sb = 0;
        for (int r = 0; r < ng; r++) {
          const cplx gra = std::conj(G[size_t(a) * ng + r]);
          sa += gra * G[size_t(b) * ng + r];
          sb += gra * VW[size_t(b) * ng + r];
        }
        Ag[size_t(b) * nt + a] = sa;
        Bg[size_t(b) * nt + a] = sb;
      }
    Mg = Ag;
    if (!hz_small::lu_solve(nt, Bg, Mg, nt)) return HZ_OK;
  }
  if (!hz_small::eig(nt, Mg, w, VR, err)) {
    c->err = err;
    return HZ_OK;
  }
  const std::vector<int> pick = smallest(w, kn);
  P.assign(size_t(nt) * kn, 0.0);
  for (int q = 0; q < kn; q++)
    for (int i = 0; i < nt; i++) P[size_t(q) * nt + i] = VR[size_t(pick[size_t(q)]) * nt + i];
  std::vector<cplx> GP(size_t(ng) * kn, 0.0), Q, R;
  for (int q = 0; q < kn; q++)
    for (int i = 0; i < ng; i++) {
      cplx sacc = 0;
      for (int j = 0; j < nt; j++) sacc += G[size_t(j) * ng + i] * P[size_t(q) * nt + j];
      GP[size_t(q) * ng + i] = sacc;
    }
  hz_small::qr_thin(ng, kn, GP, Q, R);
  if (!hz_small::tri_inv_upper(kn, R)) return HZ_OK;
  // U coefficients: P R^{-1}, recycled rows scaled by D
  std::vector<cplx> PU(size_t(nt) * kn, 0.0);
  for (int q = 0; q < kn; q++)
    for (int i = 0; i < nt; i++) {
      cplx sacc = 0;
      for (int r = 0; r <= q; r++) sacc += P[size_t(r) * nt + i] * R[size_t(q) * kn + r];
      PU[size_t(q) * nt + i] = (i < kk ? dsc[size_t(i)] : 1.0) * sacc;
    }
  TRY(combo_cols(c, {{Cb, ng}}, Q, kn, c->Ctmp, 1.0, false));                   // C = [C, V] Q
  TRY(combo_cols(c, {{c->Uh, kk}, {V, kc}}, PU, kn, c->Uht, 1.0, false));      // Uh = [Uh D, V] P R^-1
  TRY(combo_cols(c, {{c->Ux, kk}, {Z, kc}}, PU, kn, c->Uxt, 1.0, false));      // Ux = [Ux D, Z] P R^-1
  CU(cudaMemcpyAsync(V - int64_t(kn) * n, c->Ctmp, size_t(kn) * n * 16, cudaMemcpyDeviceToDevice, st));
  std::swap(c->Uh, c->Uht);
  std::swap(c->Ux, c->Uxt);
  c->rdim = kn;
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  return HZ_OK;
}

// The single right-hand side's cycle end: its Hessenberg and B columns from the device
// (Hraw: column j at j (m + 1); Braw: column j at j rk).
hz_status recycle_update(hz_ctx* c, int kk, int kc) {
  const int m = c->restart, rk = c->rk;
  if (kc < 1) return HZ_OK;
  CU(cudaStreamSynchronize(c->st));
  const std::vector<cplx> Hr = to_host(c->Hraw, size_t(m + 1) * kc);
  std::vector<cplx> Hm(size_t(kc + 1) * kc), Bm(size_t(kk) * kc);
  for (int j = 0; j < kc; j++)
    for (int i = 0; i <= kc; i++) Hm[size_t(j) * (kc + 1) + i] = Hr[size_t(j) * (m + 1) + i];
  if (kk > 0) {
    const std::vector<cplx> Bh = to_host(c->Braw, size_t(rk) * kc);
    for (int j = 0; j < kc; j++)
      for (int i = 0; i < kk; i++) Bm[size_t(j) * kk + i] = Bh[size_t(j) * rk + i];
  }
  return recycle_space(c, kk, kc, 1, Hm, Bm, c->V, c->Zs);
}

// One right-hand side by GCRO-DR (x0 = 0), with the stopping and counting rules of
// fgmres_one; the recycled space left by the previous right-hand side is used from the
// first cycle on.
hz_status block_orthonormalise(hz_ctx* c, double2* W, int s, double2* Q, std::vector<cplx>& R, const double* w0,
                               bool& brk);

// Carries the recycled space over to a new operator (options.recycle_keep, after a new
// hz_factor): C' = A Ux is orthonormalised column by column (CGS2), C' = Q R, and the space
// becomes (Ux R^{-1}, Uh R^{-1}, Q), so that C = A Ux and C^H C = I hold for the new A
// (Parks et al. 2006, for a sequence of matrices).  A numerically dependent C' drops the
// space.
hz_status recycle_rebase(hz_ctx* c) {
  const int64_t n = c->n;
  const int kk = c->rdim;
  cudaStream_t st = c->st;
  for (int i = 0; i < kk; i++)
    hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, c->Ux + int64_t(i) * n, nullptr, c->Ctmp + int64_t(i) * n, st);
  std::vector<double> w0(kk);
  for (int i = 0; i < kk; i++) TRY(norm2(c, c->Ctmp + int64_t(i) * n, w0[i]));
  std::vector<cplx> R;
  bool brk = false;
  TRY(block_orthonormalise(c, c->Ctmp, kk, recycle_basis(c) - int64_t(kk) * n, R, w0.data(), brk));
  if (brk || !hz_small::tri_inv_upper(kk, R)) {
    c->rdim = 0;
    return HZ_OK;
  }
  combo(c, kk, c->Ux, 0, nullptr, R, kk, c->Uxt, 1.0, false);      // Ux R^{-1}
  combo(c, kk, c->Uh, 0, nullptr, R, kk, c->Uht, 1.0, false);      // Uh R^{-1}
  std::swap(c->Ux, c->Uxt);
  std::swap(c->Uh, c->Uht);
  CU(cudaStreamSynchronize(st));
  return HZ_OK;
}

hz_status gcrodr_one(hz_ctx* c, double tol, hz_rhs_info* info) {
  const int64_t n = c->n;
  const int m = c->restart;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  double bnorm = 0;
  TRY(norm2(c, c->b, bnorm));
  CU(cudaMemsetAsync(c->x, 0, size_t(n) * 16, st));
  info->iterations = 0;
  info->status = HZ_OK;
  info->rel_residual = 0.0;
  if (bnorm == 0.0) return HZ_OK;
  if (!std::isfinite(bnorm)) {
    info->status = HZ_ERR_BREAKDOWN;
    return HZ_OK;
  }
  if (c->recycle_stale) {                   // the space was built for the previous operator
    c->recycle_stale = false;
    if (c->rdim > 0) TRY(recycle_rebase(c));
  }
  c->h_pin[6] = bnorm;
  CU(cudaMemcpyAsync(c->scal + 4, c->h_pin + 6, sizeof(double), cudaMemcpyHostToDevice, st));
  hz::launch_axpby_copy(n, c->b, c->w, st);                                   // r = b
  int its = 0;
  bool in_span = false;
  for (;;) {
    const int kk = c->rdim;
    c->ckk = kk;
    if (kk > 0) {
      // r orthogonal to C: x += Ux C^H r, r -= C C^H r
      const double2* Cb = c->V - int64_t(kk) * n;
      hz::launch_cgs(n, kk, Cb, n, nullptr, c->w, kk, c->partial, st);
      hz::launch_reduce(c->partial, nb, kk, c->h1, st);
      hz::launch_cgs(n, kk, Cb, n, c->h1, c->w, 0, c->partial, st);
      hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
      hz::launch_combo(n, kk, c->Ux, n, 0, nullptr, n, c->h1, 1, c->x, n, 1.0, true, st);
      // b (or the restart residual) inside span(C): x is already the solution
      CU(cudaMemcpyAsync(c->h_pin + 5, &c->nrm[64].x, sizeof(double), cudaMemcpyDeviceToHost, st));
      CU(cudaStreamSynchronize(st));
      if (std::sqrt(c->h_pin[5]) <= 1e-3 * tol * bnorm && !in_span) {
        hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, c->x, c->b, c->w, st);
        double rn = 0;
        TRY(norm2(c, c->w, rn));
        info->iterations = its;
        info->rel_residual = rn / bnorm;
        if (rn / bnorm <= tol) return HZ_OK;
        in_span = true;                     // project the true residual once more, then iterate
        continue;
      }
    } else {
      hz::launch_cgs(n, 0, c->V, n, nullptr, c->w, 0, c->partial, st);
      hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
    }
    hz::launch_init_cycle(c->nrm, c->g, m, c->scal + 2, c->scal + 3, st);
    hz::launch_scale(n, c->w, c->scal + 2, c->V, st);
    const int p = m - kk;
    int k = 0;
    bool stop_nonfinite = false;
    for (int j = 0; j < p; j++) {
      TRY(run_iteration(c, j));
      its++;
      k = j + 1;
      const double est = c->h_pin[0];
      int brk = 0;
      std::memcpy(&brk, c->h_pin + 4, sizeof(int));
      if (!std::isfinite(est)) { stop_nonfinite = true; break; }
      if (brk || est <= tol || its >= c->max_iter) break;
    }
    if (stop_nonfinite) {
      info->iterations = its;
      info->status = HZ_ERR_BREAKDOWN;
      info->rel_residual = NAN;
      return HZ_OK;
    }
    hz::launch_update_x(n, k, c->H, m + 1, c->g, c->ysol, c->Zs, n, c->x, st);   // x += Z y
    if (kk > 0) {                                                                // x -= Ux (B y)
      CU(cudaStreamSynchronize(st));
      const std::vector<cplx> y = to_host(c->ysol, size_t(k));
      const std::vector<cplx> Bh = to_host(c->Braw, size_t(c->rk) * k);
      std::vector<cplx> t(size_t(kk), 0.0);
      for (int i = 0; i < kk; i++)
        for (int j = 0; j < k; j++) t[size_t(i)] += Bh[size_t(j) * c->rk + i] * y[size_t(j)];
      combo(c, kk, c->Ux, 0, nullptr, t, 1, c->x, -1.0, true);
    }
    hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, c->x, c->b, c->w, st);          // r = b - A x
    double rn = 0;
    TRY(norm2(c, c->w, rn));
    const double rel = rn / bnorm;
    info->iterations = its;
    info->rel_residual = rel;
    if (!std::isfinite(rel)) {
      info->status = HZ_ERR_BREAKDOWN;
      return HZ_OK;
    }
    TRY(recycle_update(c, kk, k));          // kept for the next cycle and right-hand side
    if (rel <= tol) return HZ_OK;
    if (its >= c->max_iter) {
      info->status = HZ_ERR_NOT_CONVERGED;
      return HZ_OK;
    }
  }
}

// ---------------------------------------------------------------------------
// Pseudo-block FGMRES: S slots, each holding one right-hand side with its own Krylov
// space, Givens rotations, cycle position and stopping decisions (the recurrence of
// fgmres_one).  Every preconditioner and operator application works on the S vectors
// at once (interleaved per row), so each factor panel is read once for S right-hand
// sides; a slot whose solve ends takes new work while the others continue.
// ---------------------------------------------------------------------------
void apply_prec_multi(hz_ctx* c, const double2* X, double2* Y) {
  const int S = c->S;
  cudaStream_t st = c->st;
  if (c->levels == 2) {
    hz::launch_spmv_real_multi(c->nH, S, c->d_Ztrp, c->d_Ztci, c->d_Ztv, X, c->rHi, st);   // Z^T v
    if (c->coarse_oras) {                                                                 // E^{-1}
      // one inner solve per running slot (each right-hand side has its own coarse problem)
      cudaMemsetAsync(c->yHi, 0, size_t(S) * c->nH * 16, st);
      for (int i = 0; i < S; i++) {
        if (c->slots[i].state != hz_ctx::SLOT_RUN) continue;
        hz::SlotCols one;
        for (int q = 0; q < 16; q++) one.o[q] = q == i ? 0 : -1;
        hz::launch_deinterleave(c->nH, S, one, c->rHi, c->rH, st);
        coarse_inner(c, c->rH, c->yH);
        hz::launch_interleave_put(c->nH, S, i, c->yH, c->yHi, st);
      }
    } else {
      hz::launch_local_multi(c->crs, S, c->rHi, nullptr, c->yHi, st);
    }
    hz::launch_spmv_real_multi(c->n, S, c->d_Zrp, c->d_Zci, c->d_Zv, c->yHi, c->yi, st);  // y = Z y_H
    hz::launch_spmv_multi(c->n, S, c->d_rp, c->d_ci, c->d_A, c->yi, X, c->Ti, st);         // t = v - A y
    hz::launch_local_multi(c->loc, S, c->Ti, c->yi, Y, st);                               // y + M_1^{-1} t
  } else {
    hz::launch_local_multi(c->loc, S, X, nullptr, Y, st);
  }
}

double2* slot_V(hz_ctx* c, int i) { return c->Vb + int64_t(i) * c->n * (c->restart + 1); }
double2* slot_Z(hz_ctx* c, int i) { return c->Zb + int64_t(i) * c->n * c->restart; }
double2* slot_col(hz_ctx* c, double2* base, int i) { return base + int64_t(i) * c->n; }
double* slot_scal(hz_ctx* c, int i) { return c->scalb + int64_t(i) * 8; }

// New cycle of slot i from the residual in Wc[i] (|r|^2 in nrm): g = beta e_1, v_0 = r / beta.
void slot_cycle(hz_ctx* c, int i) {
  const int m = c->restart;
  hz::launch_init_cycle(c->nrm, c->gb + int64_t(i) * (m + 1), m, slot_scal(c, i) + 2, slot_scal(c, i) + 3, c->st);
  hz::launch_scale(c->n, slot_col(c, c->Wc, i), slot_scal(c, i) + 2, slot_V(c, i), c->st);
  c->slots[i].j = 0;
}

}  // namespace

namespace hz_engine {

// Starts the right-hand side already in Bc[i] with x0 = 0 (r = b).
hz_status slot_start(hz_ctx* c, int i, double tol, int64_t tag) {
  hz_ctx::Slot& s = c->slots[i];
  s = hz_ctx::Slot{};
  s.tag = tag;
  s.tol = tol;
  s.state = hz_ctx::SLOT_RUN;
  CU(cudaMemsetAsync(slot_col(c, c->Xc, i), 0, size_t(c->n) * 16, c->st));
  TRY(norm2(c, slot_col(c, c->Bc, i), s.bnorm));        // leaves |b|^2 in nrm
  if (s.bnorm == 0.0) {
    s.state = hz_ctx::SLOT_DONE;
    return HZ_OK;
  }
  if (!std::isfinite(s.bnorm)) {
    s.state = hz_ctx::SLOT_DONE;
    s.info.status = HZ_ERR_BREAKDOWN;
    s.info.rel_residual = NAN;
    return HZ_OK;
  }
  c->h_pin[hz_ctx::PIN_BNORM + i] = s.bnorm;             // |b| for the Givens breakdown test
  CU(cudaMemcpyAsync(slot_scal(c, i) + 4, c->h_pin + hz_ctx::PIN_BNORM + i, sizeof(double),
                     cudaMemcpyHostToDevice, c->st));
  hz::launch_axpby_copy(c->n, slot_col(c, c->Bc, i), slot_col(c, c->Wc, i), c->st);
  slot_cycle(c, i);
  return HZ_OK;
}

// Right-hand side of one point source (Eq. 2 load -phi_a(x_s)) written into Bc[i].
hz_status slot_point_source(hz_ctx* c, int i, const double xyz[3]) {
  int64_t e = -1;
  double lam[4], phi[10];
  if (!hz::locate_point(c->mesh, xyz, e, lam)) return fail(c, HZ_ERR_ARG, "source outside the mesh");
  hz::eval_basis(c->order, lam, phi);
  hz::PointRhs p{};
  for (int a = 0; a < c->dofs.nb; a++) {
    const int64_t g = c->dofs.elem[int64_t(c->dofs.nb) * e + a];
    if (c->dofs.is_dir[g]) continue;
    p.idx[p.cnt] = g;
    p.val[p.cnt] = -phi[a];
    p.cnt++;
  }
  CU(cudaMemsetAsync(slot_col(c, c->Bc, i), 0, size_t(c->n) * 16, c->st));
  hz::launch_point_rhs(p, slot_col(c, c->Bc, i), c->st);
  return HZ_OK;
}

// Enqueues one inner iteration of every running slot (no host wait): the batched
// z_j = M^{-1} v_j and w = A z_j over all S slots, then per slot CGS2 against its own
// basis, the Givens update at its own position j and v_{j+1}; the per-slot residual
// estimates and breakdown flags are copied to pinned memory.
void slots_issue(hz_ctx* c) {
  const int S = c->S, m = c->restart;
  const int64_t n = c->n;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  if (c->spmv_lanes) hz::set_spmv_lanes(c->spmv_lanes);
  hz::SlotCols vin, zout, wout;
  for (int i = 0; i < 16; i++) vin.o[i] = zout.o[i] = wout.o[i] = -1;
  for (int i = 0; i < S; i++) {
    const hz_ctx::Slot& s = c->slots[i];
    if (s.state != hz_ctx::SLOT_RUN) continue;
    vin.o[i] = int64_t(i) * n * (m + 1) + int64_t(s.j) * n;
    zout.o[i] = int64_t(i) * n * m + int64_t(s.j) * n;
    wout.o[i] = int64_t(i) * n;
  }
  hz::launch_interleave(n, S, vin, c->Vb, c->Xi, st);
  apply_prec_multi(c, c->Xi, c->Yi);
  hz::launch_deinterleave(n, S, zout, c->Yi, c->Zb, st);
  hz::launch_spmv_multi(n, S, c->d_rp, c->d_ci, c->d_A, c->Yi, nullptr, c->Wi, st);
  hz::launch_deinterleave(n, S, wout, c->Wi, c->Wc, st);
  // CGS2 against each slot's own basis, the Givens update at its own j and v_{j+1},
  // every step one launch for all slots
  hz::SlotCgs pc{};
  hz::SlotGivens pg{};
  hz::SlotScale ps{};
  pg.m = m;
  pg.H = c->Hb;
  pg.sn = c->snb;
  pg.g = c->gb;
  pg.cs = c->csb;
  pg.h1 = c->h1s;
  pg.h2 = c->h2s;
  pg.nrm = c->nrms;
  pg.scal = c->scalb;
  pg.brk = c->brkb;
  for (int i = 0; i < 16; i++) {
    const bool run = i < S && c->slots[i].state == hz_ctx::SLOT_RUN;
    const int j = run ? c->slots[i].j : -1;
    pc.V[i] = run ? slot_V(c, i) : nullptr;
    pc.w[i] = run ? slot_col(c, c->Wc, i) : nullptr;
    pc.h[i] = c->h1s + int64_t(i) * 65;
    pc.ncols[i] = run ? j + 1 : -1;
    pg.j[i] = j;
    ps.w[i] = pc.w[i];
    ps.s[i] = run ? slot_scal(c, i) + 1 : nullptr;
    ps.out[i] = run ? slot_V(c, i) + int64_t(j + 1) * n : nullptr;
  }
  hz::launch_cgs_slots(n, S, pc, false, true, c->partial_s, c->h1s, st);    // h1 = V^H w
  hz::launch_cgs_slots(n, S, pc, true, true, c->partial_s, c->h2s, st);     // w -= V h1; h2 = V^H w
  for (int i = 0; i < 16; i++) pc.h[i] = c->h2s + int64_t(i) * 65;
  hz::launch_cgs_slots(n, S, pc, true, false, c->partial_s, c->nrms, st);   // w -= V h2; |w|^2
  hz::launch_givens_slots(S, pg, st);
  hz::launch_scale_slots(n, S, ps, st);
  cudaMemcpyAsync(c->h_pin + hz_ctx::PIN_SLOT, c->scalb, size_t(S) * 8 * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(c->h_pin + hz_ctx::PIN_FLAGS, c->brkb, size_t(S) * sizeof(int), cudaMemcpyDeviceToHost, st);
}

// End of slot i's cycle: x += Z y, true residual ||b - A x|| / ||b||; the slot either
// finishes (converged, iteration limit, non-finite) or restarts from that residual.
static hz_status slot_end_cycle(hz_ctx* c, int i) {
  hz_ctx::Slot& s = c->slots[i];
  const int m = c->restart;
  const int64_t n = c->n;
  double2* xi = slot_col(c, c->Xc, i);
  hz::launch_update_x(n, s.j, c->Hb + int64_t(i) * (m + 1) * m, m + 1, c->gb + int64_t(i) * (m + 1),
                      c->yb + int64_t(i) * m, slot_Z(c, i), n, xi, c->st);
  hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, xi, slot_col(c, c->Bc, i), slot_col(c, c->Wc, i), c->st);
  double rn = 0;
  TRY(norm2(c, slot_col(c, c->Wc, i), rn));             // leaves |r|^2 in nrm for a restart
  const double rel = rn / s.bnorm;
  s.info.iterations = s.its;
  s.info.rel_residual = rel;
  if (!std::isfinite(rel)) {
    s.info.status = HZ_ERR_BREAKDOWN;
    s.state = hz_ctx::SLOT_DONE;
  } else if (rel <= s.tol) {
    s.state = hz_ctx::SLOT_DONE;
  } else if (s.its >= c->max_iter) {
    s.info.status = HZ_ERR_NOT_CONVERGED;
    s.state = hz_ctx::SLOT_DONE;
  } else {
    slot_cycle(c, i);
  }
  return HZ_OK;
}

// Waits for the step issued by slots_issue and applies each running slot's stopping
// decisions (the rule of fgmres_one, per slot).
hz_status slots_complete(hz_ctx* c) {
  CU(cudaStreamSynchronize(c->st));
  CU(cudaGetLastError());
  const double* hs = c->h_pin + hz_ctx::PIN_SLOT;
  const int* hb = reinterpret_cast<const int*>(c->h_pin + hz_ctx::PIN_FLAGS);
  if (c->spmv_lanes) hz::set_spmv_lanes(c->spmv_lanes);
  for (int i = 0; i < c->S; i++) {
    hz_ctx::Slot& s = c->slots[i];
    if (s.state != hz_ctx::SLOT_RUN) continue;
    s.its++;
    s.j++;
    const double est = hs[8 * i];
    if (!std::isfinite(est)) {
      s.state = hz_ctx::SLOT_DONE;
      s.info.iterations = s.its;
      s.info.status = HZ_ERR_BREAKDOWN;
      s.info.rel_residual = NAN;
      continue;
    }
    if (hb[i] || est <= s.tol || s.its >= c->max_iter || s.j == c->restart) TRY(slot_end_cycle(c, i));
  }
  return HZ_OK;
}

int slot_count(const hz_ctx* c) { return c->S; }
void slot_reset(hz_ctx* c, int i) { c->slots[i] = hz_ctx::Slot{}; }
int slot_state(const hz_ctx* c, int i) { return c->slots[i].state; }
bool slots_running(const hz_ctx* c) {
  for (int i = 0; i < c->S; i++)
    if (c->slots[i].state == hz_ctx::SLOT_RUN) return true;
  return false;
}

// Copies a finished slot's solution (device or host destination) and frees the slot.
hz_status slot_harvest(hz_ctx* c, int i, void* x, bool on_device, hz_rhs_info* info) {
  hz_ctx::Slot& s = c->slots[i];
  if (s.state != hz_ctx::SLOT_DONE) return fail(c, HZ_ERR_STATE, "slot has no finished solve");
  CU(cudaMemcpyAsync(x, slot_col(c, c->Xc, i), size_t(c->n) * 16,
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  CU(cudaStreamSynchronize(c->st));
  if (info) *info = s.info;
  s = hz_ctx::Slot{};
  return HZ_OK;
}

}  // namespace hz_engine

namespace {

// Pseudo-block solve of nrhs right-hand sides through the S slots: a slot whose solve
// ends takes the next right-hand side at once, so the slots stay full.
hz_status solve_slots(hz_ctx* c, const double2* rhs, int nrhs, double tol, double2* x, bool on_device,
                      hz_rhs_info* info, hz_status& worst) {
  const int64_t n = c->n;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (auto& s : c->slots) s = hz_ctx::Slot{};
  int next = 0, left = nrhs;
  while (left > 0) {
    for (int i = 0; i < c->S && next < nrhs; i++) {
      if (c->slots[i].state != hz_ctx::SLOT_FREE) continue;
      CU(cudaMemcpyAsync(slot_col(c, c->Bc, i), rhs + int64_t(next) * n, size_t(n) * 16, kin, c->st));
      TRY(hz_engine::slot_start(c, i, tol, next));
      next++;
    }
    if (hz_engine::slots_running(c)) {
      hz_engine::slots_issue(c);
      TRY(hz_engine::slots_complete(c));
    }
    for (int i = 0; i < c->S; i++) {
      if (c->slots[i].state != hz_ctx::SLOT_DONE) continue;
      const int64_t k = c->slots[i].tag;
      hz_rhs_info inf{};
      TRY(hz_engine::slot_harvest(c, i, x + k * n, on_device, &inf));
      if (info) info[k] = inf;
      if (inf.status != HZ_OK && worst == HZ_OK) worst = hz_status(inf.status);
      left--;
    }
  }
  return HZ_OK;
}

// ---------------------------------------------------------------------------
// Block FGMRES (krylov == HZ_KRYLOV_BLOCK): one block Krylov space for s <= S
// right-hand sides.  The steps are those of the oracle's block_fgmres:
//   * the residual block is factored column by column (CGS2 against the block's
//     earlier columns) into V_0 and the upper-triangular beta;
//   * block step j: Z_j = M^{-1} V_j and W = A Z_j on the interleaved slot operators;
//     two classical Gram-Schmidt passes of the s columns against V_0..V_j, in chunks of
//     64 basis columns (all chunks' coefficients before any update), then the columns
//     of W orthonormalised among themselves into V_{j+1};
//   * the band Hessenberg matrix is reduced by Givens rotations on the host (each
//     between the diagonal row and one of the s rows below it, bottom row first), the
//     same rotations are applied to G = [beta; 0], and the estimate of right-hand side i
//     is the norm of column i of G's rows below the triangle;
//   * the cycle ends when every estimate / ||b_i|| <= tol, on a happy breakdown or at
//     max_iter; x += Z R^{-1} G_top; the true residuals are checked and the next cycle
//     restarts from them.
// Device storage is the slot engine's: V = Vb as one n x (m + 1) S block, Z = Zb,
// W = Wc, B = Bc, X = Xc.  The host waits once per column of the per-block
// orthonormalisation, so block steps run as eager launches.
// ---------------------------------------------------------------------------
hz_status block_orthonormalise(hz_ctx* c, double2* W, int s, double2* Q, std::vector<cplx>& R, const double* w0,
                               bool& brk) {
  const int64_t n = c->n;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  R.assign(size_t(s) * s, cplx(0.0, 0.0));
  brk = false;
  std::vector<double2> hh(3 * 65);
  for (int q = 0; q < s; q++) {
    double2* w = W + int64_t(q) * n;
    if (q > 0) {
      hz::launch_cgs(n, q, Q, n, nullptr, w, q, c->partial, st);
      hz::launch_reduce(c->partial, nb, q, c->h1, st);
      hz::launch_cgs(n, q, Q, n, c->h1, w, q, c->partial, st);
      hz::launch_reduce(c->partial, nb, q, c->h2, st);
      hz::launch_cgs(n, q, Q, n, c->h2, w, 0, c->partial, st);
    } else {
      hz::launch_cgs(n, 0, Q, n, nullptr, w, 0, c->partial, st);
    }
    hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
    CU(cudaMemcpyAsync(hh.data(), c->h1, 65 * 16, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(hh.data() + 65, c->h2, 65 * 16, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(hh.data() + 130, c->nrm, 65 * 16, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (int i = 0; i < q; i++) R[i + size_t(q) * s] = cplx(hh[i].x + hh[65 + i].x, hh[i].y + hh[65 + i].y);
    const double nr = std::sqrt(hh[130 + 64].x);
    R[q + size_t(q) * s] = nr;
    if (!(nr > 1e-14 * w0[q])) brk = true;
    c->h_pin[6] = nr > 0.0 ? 1.0 / nr : 0.0;
    CU(cudaMemcpyAsync(c->scal + 6, c->h_pin + 6, sizeof(double), cudaMemcpyHostToDevice, st));
    hz::launch_scale(n, w, c->scal + 6, Q + int64_t(q) * n, st);
  }
  CU(cudaStreamSynchronize(st));
  return HZ_OK;
}

// Block step j: Z_j = M^{-1} V_j, W = A Z_j, block CGS2 against [C, V_0..V_j] (C: the kk
// recycled columns stored right before V; kk = 0 without recycling) and the new block.
// hcol ((kk + (j + 2) s) x s, column-major, host): rows [0, kk) the coefficients against C,
// then the step's column of the block Hessenberg matrix.
hz_status block_step(hz_ctx* c, int j, int s, int kk, std::vector<cplx>& hcol, bool& brk) {
  const int S = c->S;
  const int64_t n = c->n;
  cudaStream_t st = c->st;
  hz::SlotCols vin, zout, wout;
  for (int i = 0; i < 16; i++) vin.o[i] = zout.o[i] = wout.o[i] = -1;
  for (int i = 0; i < s; i++) {
    vin.o[i] = int64_t(j * s + i) * n;
    zout.o[i] = int64_t(j * s + i) * n;
    wout.o[i] = int64_t(i) * n;
  }
  hz::launch_interleave(n, S, vin, c->Vb, c->Xi, st);
  apply_prec_multi(c, c->Xi, c->Yi);
  hz::launch_deinterleave(n, S, zout, c->Yi, c->Zb, st);
  hz::launch_spmv_multi(n, S, c->d_rp, c->d_ci, c->d_A, c->Yi, nullptr, c->Wi, st);
  hz::launch_deinterleave(n, S, wout, c->Wi, c->Wc, st);
  std::vector<double> w0(s);
  for (int i = 0; i < s; i++) TRY(norm2(c, c->Wc + int64_t(i) * n, w0[i]));
  const double2* base = c->Vb - int64_t(kk) * n;
  const int p = kk + (j + 1) * s;
  const int nch = (p + 63) / 64;
  hz::SlotCgs pc{};
  for (int pass = 0; pass < 2; pass++) {
    for (int k = 0; k < nch; k++) {
      for (int i = 0; i < 16; i++) {
        const bool on = i < s;
        pc.V[i] = on ? base + int64_t(64) * k * n : nullptr;
        pc.w[i] = on ? c->Wc + int64_t(i) * n : nullptr;
        pc.h[i] = nullptr;
        pc.ncols[i] = on ? std::min(64, p - 64 * k) : -1;
      }
      hz::launch_cgs_slots(n, S, pc, false, true, c->partial_s, c->hblk + (int64_t(pass) * nch + k) * S * 65, st);
    }
    for (int k = 0; k < nch; k++) {
      for (int i = 0; i < 16; i++) {
        const bool on = i < s;
        pc.V[i] = on ? base + int64_t(64) * k * n : nullptr;
        pc.w[i] = on ? c->Wc + int64_t(i) * n : nullptr;
        pc.h[i] = on ? c->hblk + ((int64_t(pass) * nch + k) * S + i) * 65 : nullptr;
        pc.ncols[i] = on ? std::min(64, p - 64 * k) : -1;
      }
      hz::launch_cgs_slots(n, S, pc, true, false, c->partial_s, c->nrms, st);
    }
  }
  std::vector<double2> hb(size_t(2) * nch * S * 65);
  CU(cudaMemcpyAsync(hb.data(), c->hblk, hb.size() * 16, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const int ld = p + s;
  hcol.assign(size_t(ld) * s, cplx(0.0, 0.0));
  for (int i = 0; i < s; i++)
    for (int r = 0; r < p; r++) {
      const int k = r / 64, jj = r % 64;
      const double2 a = hb[((size_t(0) * nch + k) * S + i) * 65 + jj];
      const double2 b = hb[((size_t(1) * nch + k) * S + i) * 65 + jj];
      hcol[r + size_t(i) * ld] = cplx(a.x + b.x, a.y + b.y);
    }
  std::vector<cplx> R;
  TRY(block_orthonormalise(c, c->Wc, s, c->Vb + int64_t(p - kk) * n, R, w0.data(), brk));
  for (int i = 0; i < s; i++)
    for (int r = 0; r < s; r++) hcol[p + r + size_t(i) * ld] = R[r + size_t(i) * s];
  return HZ_OK;
}

// Solves the s right-hand sides in Bc[0..s) (all nonzero) into Xc[0..s).  With recycling
// (options.recycle = rk > 0) this is block GCRO-DR: each cycle first makes the residual
// block orthogonal to C (X += Ux C^H R, R -= C C^H R), runs at most m - ceil(kk / s) block
// steps against [C, V], adds X += Z Y - Ux (B Y), and replaces the recycled space by the
// cycle's block harmonic Ritz vectors; the space is kept for the next batch.
hz_status block_batch(hz_ctx* c, int s, double tol, hz_rhs_info* info) {
  const int64_t n = c->n;
  const int m = c->restart;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  for (int i = 0; i < c->S; i++) c->slots[i].state = i < s ? hz_ctx::SLOT_RUN : hz_ctx::SLOT_FREE;
  std::vector<double> bn(s), rel(s, 0.0);
  for (int i = 0; i < s; i++) TRY(norm2(c, c->Bc + int64_t(i) * n, bn[i]));
  CU(cudaMemsetAsync(c->Xc, 0, size_t(s) * n * 16, st));
  CU(cudaMemcpyAsync(c->Wc, c->Bc, size_t(s) * n * 16, cudaMemcpyDeviceToDevice, st));
  const int ldh = (m + 1) * s;
  std::vector<cplx> H, Hr, Bm, G, hcol, beta;
  struct Rot { int i, r; double cs; cplx sn; };
  std::vector<Rot> rots;
  auto givens = [](cplx a, cplx b, double& cs, cplx& sn) {
    const double aa = std::abs(a);
    if (aa == 0.0) { cs = 0.0; sn = cplx(1.0, 0.0); return; }
    const double rho = std::sqrt(aa * aa + std::norm(b));
    cs = aa / rho;
    sn = (a / aa) * std::conj(b) / rho;
  };
  int its = 0;
  bool nonfinite = false;
  for (;;) {
    const int kk = c->rk > 0 ? c->rdim : 0;
    if (kk > 0) {
      const double2* Cb = c->Vb - int64_t(kk) * n;
      for (int i = 0; i < s; i++) {
        double2* wi = c->Wc + int64_t(i) * n;
        hz::launch_cgs(n, kk, Cb, n, nullptr, wi, kk, c->partial, st);
        hz::launch_reduce(c->partial, nb, kk, c->h1, st);
        hz::launch_cgs(n, kk, Cb, n, c->h1, wi, 0, c->partial, st);
        hz::launch_combo(n, kk, c->Ux, n, 0, nullptr, n, c->h1, 1, c->Xc + int64_t(i) * n, n, 1.0, true, st);
      }
    }
    std::vector<double> rn(s);
    for (int i = 0; i < s; i++) TRY(norm2(c, c->Wc + int64_t(i) * n, rn[i]));
    bool brk0 = false;
    TRY(block_orthonormalise(c, c->Wc, s, c->Vb, beta, rn.data(), brk0));
    const int psteps = std::max(1, m - (kk + s - 1) / s);
    H.assign(size_t(ldh) * m * s, cplx(0.0, 0.0));
    Hr.assign(H.size(), cplx(0.0, 0.0));                       // unrotated copy
    Bm.assign(size_t(kk) * m * s, cplx(0.0, 0.0));
    G.assign(size_t(ldh) * s, cplx(0.0, 0.0));
    for (int i = 0; i < s; i++)
      for (int r = 0; r <= i; r++) G[r + size_t(i) * ldh] = beta[r + size_t(i) * s];
    rots.clear();
    int k = 0;
    for (int j = 0; j < psteps; j++) {
      bool brk = false;
      TRY(block_step(c, j, s, kk, hcol, brk));
      const int lc = kk + (j + 2) * s;
      for (int q = 0; q < s; q++) {
        for (int r = 0; r < kk; r++) Bm[r + size_t(j * s + q) * kk] = hcol[r + size_t(q) * lc];
        for (int r = 0; r < (j + 2) * s; r++)
          H[r + size_t(j * s + q) * ldh] = Hr[r + size_t(j * s + q) * ldh] = hcol[kk + r + size_t(q) * lc];
      }
      for (int q = 0; q < s; q++) {
        const int col = j * s + q;
        cplx* hc = H.data() + size_t(col) * ldh;
        for (const Rot& g : rots) {
          const cplx t = g.cs * hc[g.i] + g.sn * hc[g.r];
          hc[g.r] = -std::conj(g.sn) * hc[g.i] + g.cs * hc[g.r];
          hc[g.i] = t;
        }
        for (int r = col + s; r > col; r--) {               // bottom row first
          double cs;
          cplx sn;
          givens(hc[col], hc[r], cs, sn);
          hc[col] = cs * hc[col] + sn * hc[r];
          hc[r] = 0.0;
          for (int i = 0; i < s; i++) {
            cplx* gi = G.data() + size_t(i) * ldh;
            const cplx t = cs * gi[col] + sn * gi[r];
            gi[r] = -std::conj(sn) * gi[col] + cs * gi[r];
            gi[col] = t;
          }
          rots.push_back({col, r, cs, sn});
        }
      }
      its++;
      k = j + 1;
      bool all = true;
      for (int i = 0; i < s; i++) {
        double e = 0.0;
        for (int r = k * s; r < (k + 1) * s; r++) e += std::norm(G[r + size_t(i) * ldh]);
        const double est = std::sqrt(e) / bn[i];
        if (!std::isfinite(est)) nonfinite = true;
        all = all && est <= tol;
      }
      if (brk || all || nonfinite || its >= c->max_iter) break;
    }
    // Y = R^{-1} G_top, x += Z Y (64 columns of Z at a time)
    const int p = k * s;
    std::vector<cplx> Y(size_t(p) * s);
    for (int i = 0; i < s; i++)
      for (int r = p - 1; r >= 0; r--) {
        cplx acc = G[r + size_t(i) * ldh];
        for (int l = r + 1; l < p; l++) acc -= H[r + size_t(l) * ldh] * Y[l + size_t(i) * p];
        Y[r + size_t(i) * p] = acc / H[r + size_t(r) * ldh];
      }
    CU(cudaMemcpyAsync(c->yblk, Y.data(), Y.size() * 16, cudaMemcpyHostToDevice, st));
    for (int i = 0; i < s; i++)
      for (int q0 = 0; q0 < p; q0 += 64)
        hz::launch_gemv_add(n, std::min(64, p - q0), c->yblk + size_t(i) * p + q0, c->Zb + int64_t(q0) * n, n,
                            c->Xc + int64_t(i) * n, st);
    if (kk > 0) {                                              // X -= Ux (B Y)
      std::vector<cplx> T(size_t(kk) * s, 0.0);
      for (int i = 0; i < s; i++)
        for (int l = 0; l < p; l++)
          for (int r = 0; r < kk; r++) T[r + size_t(i) * kk] += Bm[r + size_t(l) * kk] * Y[l + size_t(i) * p];
      combo(c, kk, c->Ux, 0, nullptr, T, s, c->Xc, -1.0, true);
    }
    // true residuals (into W, the next cycle's residual block)
    bool done = true;
    for (int i = 0; i < s; i++) {
      hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, c->Xc + int64_t(i) * n, c->Bc + int64_t(i) * n,
                      c->Wc + int64_t(i) * n, st);
      double r;
      TRY(norm2(c, c->Wc + int64_t(i) * n, r));
      rel[i] = r / bn[i];
      if (!std::isfinite(rel[i])) nonfinite = true;
      done = done && rel[i] <= tol;
    }
    if (c->rk > 0 && !nonfinite) {                             // the cycle's block harmonic Ritz space
      std::vector<cplx> Hm(size_t(p + s) * p), Bp(size_t(kk) * p);
      for (int l = 0; l < p; l++) {
        for (int r = 0; r < p + s; r++) Hm[r + size_t(l) * (p + s)] = Hr[r + size_t(l) * ldh];
        for (int r = 0; r < kk; r++) Bp[r + size_t(l) * kk] = Bm[r + size_t(l) * kk];
      }
      TRY(recycle_space(c, kk, p, s, Hm, Bp, c->Vb, c->Zb));
    }
    if (done || nonfinite || its >= c->max_iter) break;
  }
  for (int i = 0; i < s; i++) {
    info[i].iterations = its;
    info[i].rel_residual = rel[i];
    info[i].status = nonfinite ? HZ_ERR_BREAKDOWN : (rel[i] <= tol ? HZ_OK : HZ_ERR_NOT_CONVERGED);
  }
  for (int i = 0; i < c->S; i++) c->slots[i].state = hz_ctx::SLOT_FREE;
  return HZ_OK;
}

// Block FGMRES (block GCRO-DR with recycling) over nrhs right-hand sides in batches of S;
// zero columns get x = 0.
hz_status solve_block(hz_ctx* c, const double2* rhs, int nrhs, double tol, double2* x, bool on_device,
                      hz_rhs_info* info, hz_status& worst) {
  const int64_t n = c->n;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (c->recycle_stale) {                   // the space was built for the previous operator
    c->recycle_stale = false;
    if (c->rdim > 0) TRY(recycle_rebase(c));
  }
  int next = 0;
  while (next < nrhs) {
    std::vector<int> cols;
    while (next < nrhs && int(cols.size()) < c->S) {
      const int k = next++;
      CU(cudaMemcpyAsync(c->Bc + int64_t(cols.size()) * n, rhs + int64_t(k) * n, size_t(n) * 16, kin, c->st));
      double bnorm;
      TRY(norm2(c, c->Bc + int64_t(cols.size()) * n, bnorm));
      if (bnorm == 0.0) {                                    // x = 0, no iteration
        CU(cudaMemsetAsync(c->w, 0, size_t(n) * 16, c->st));
        CU(cudaMemcpyAsync(x + int64_t(k) * n, c->w, size_t(n) * 16, kout, c->st));
        if (info) info[k] = hz_rhs_info{0, HZ_OK, 0.0};
        continue;
      }
      cols.push_back(k);
    }
    if (cols.empty()) continue;
    std::vector<hz_rhs_info> inf(cols.size());
    TRY(block_batch(c, int(cols.size()), tol, inf.data()));
    for (size_t i = 0; i < cols.size(); i++) {
      CU(cudaMemcpyAsync(x + int64_t(cols[i]) * n, c->Xc + int64_t(i) * n, size_t(n) * 16, kout, c->st));
      if (info) info[cols[i]] = inf[i];
      if (inf[i].status != HZ_OK && worst == HZ_OK) worst = hz_status(inf[i].status);
    }
  }
  return HZ_OK;
}

// Autotuner: lanes per row of the complex SpMV, timed on this matrix (3 runs each
// after a warm-up, CUDA events on the context stream); the fastest is kept.
hz_status tune_spmv(hz_ctx* c) {
  CU(cudaMemsetAsync(c->b, 0x3f, size_t(c->n) * 16, c->st));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int pick = 8;
  for (int t : {2, 4, 8, 16}) {
    hz::set_spmv_lanes(t);
    hz::launch_spmv(c->n, c->d_rp, c->d_ci, c->d_A, c->b, nullptr, c->w, c->st);
    CU(cudaEventRecord(e0, c->st));
    for (int r = 0; r < 3; r++) hz::launch_spmv(c->n, c->d_rp, c->d_ci, c->d_A, c->b, nullptr, c->w, c->st);
    CU(cudaEventRecord(e1, c->st));
    CU(cudaEventSynchronize(e1));
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->spmv_lanes = pick;
  return HZ_OK;
}

hz_status check_ctx(hz_ctx* c) {
  if (!c) return HZ_ERR_ARG;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return fail(c, HZ_ERR_CUDA, cudaGetErrorString(e));
  return HZ_OK;
}

}  // namespace

extern "C" {

const char* hz_status_string(hz_status s) {
  switch (s) {
    case HZ_OK: return "ok";
    case HZ_ERR_ARG: return "invalid argument";
    case HZ_ERR_STATE: return "call out of order";
    case HZ_ERR_OOM: return "out of device memory";
    case HZ_ERR_CUDA: return "CUDA error";
    case HZ_ERR_ZERO_PIVOT: return "zero pivot";
    case HZ_ERR_BREAKDOWN: return "breakdown";
    case HZ_ERR_NOT_CONVERGED: return "not converged";
    case HZ_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

const char* hz_last_error(const hz_ctx* c) { return c ? c->err.c_str() : ""; }

int64_t hz_ndofs(const hz_ctx* c) { return c ? c->n : -1; }

hz_status hz_get_stats(const hz_ctx* c, hz_stats* out) {
  if (!c || !out) return HZ_ERR_ARG;
  *out = c->stats;
  out->recycle_dim = c->rdim;
  out->device_bytes = c->bytes;
  out->launches = hz::launch_count();
  return HZ_OK;
}

void hz_free(hz_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->st) cudaStreamSynchronize(c->st);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->sizes.clear();
  for (cudaGraphExec_t g : c->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  free_host_ptrs(c->loc);
  free_host_ptrs(c->crs);
  free_host_ptrs(c->cloc);
  delete c;
}

}  // extern "C"

// Host analysis shared by hz_setup_mesh and hz_plan.  HZ_VERBOSE=1 prints phase times.
// Resident and peak host memory of this process in GB (Linux /proc; 0 elsewhere).
static void host_rss_gb(double& rss, double& peak) {
  rss = peak = 0.0;
  if (FILE* f = std::fopen("/proc/self/status", "r")) {
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
      long long kb = 0;
      if (std::sscanf(line, "VmRSS: %lld", &kb) == 1) rss = kb / 1e6;
      if (std::sscanf(line, "VmHWM: %lld", &kb) == 1) peak = kb / 1e6;
    }
    std::fclose(f);
  }
}

static void phase(const char* what, std::chrono::steady_clock::time_point& t) {
  static const bool on = std::getenv("HZ_VERBOSE") != nullptr;
  const auto now = std::chrono::steady_clock::now();
  if (on) {
    double rss, peak;
    host_rss_gb(rss, peak);
    std::fprintf(stderr, "[hz] %-28s %8.3f s   host RSS %6.2f GB (peak %6.2f)\n", what,
                 std::chrono::duration<double>(now - t).count(), rss, peak);
  }
  t = now;
}

static hz_status analyse(hz_ctx* c, const hz_mesh_desc* md, const hz_options* op, hz::HostProblem& P) {
  if (!md || !op) return fail(c, HZ_ERR_ARG, "null mesh or options");
  if (md->order != 1 && md->order != 2) return fail(c, HZ_ERR_ARG, "order must be 1 or 2");
  if (md->nv <= 0 || md->ne <= 0 || !md->xyz || !md->tets || !md->c_re || !md->c_im)
    return fail(c, HZ_ERR_ARG, "empty or incomplete mesh");
  if (md->nf > 0 && (!md->faces || !md->face_tag)) return fail(c, HZ_ERR_ARG, "faces without tags");
  if (op->nsub < 1 || op->overlap < 0 || (op->levels != 1 && op->levels != 2))
    return fail(c, HZ_ERR_ARG, "bad nsub / overlap / levels");
  if (op->restart < 1 || op->restart > 63) return fail(c, HZ_ERR_ARG, "restart must be in [1, 63]");
  if (op->precision != HZ_FP64 && op->precision != HZ_MIXED) return fail(c, HZ_ERR_ARG, "bad precision");
  if (op->spmv_lanes != 0 && op->spmv_lanes != 2 && op->spmv_lanes != 4 && op->spmv_lanes != 8 &&
      op->spmv_lanes != 16)
    return fail(c, HZ_ERR_ARG, "spmv_lanes must be 0, 2, 4, 8 or 16");
  if (op->coarse_solver != HZ_COARSE_DIRECT && op->coarse_solver != HZ_COARSE_ORAS)
    return fail(c, HZ_ERR_ARG, "bad coarse_solver");
  if (op->coarse_maxit < 0 || op->coarse_maxit > 63 || !(op->coarse_tol >= 0.0))
    return fail(c, HZ_ERR_ARG, "coarse_maxit must be in [0, 63] and coarse_tol >= 0");
  if (op->recycle < 0 || op->recycle > 16 || 2 * op->recycle > op->restart)
    return fail(c, HZ_ERR_ARG, "recycle must be in [0, min(16, restart / 2)]");
  if (op->recycle > 0 && op->block_size > 1 && op->krylov != HZ_KRYLOV_BLOCK)
    return fail(c, HZ_ERR_ARG, "recycle with block_size > 1 needs krylov = HZ_KRYLOV_BLOCK");
  if (op->sweep_tasks < 0 || op->sweep_tasks > 2) return fail(c, HZ_ERR_ARG, "sweep_tasks must be 0, 1 or 2");
  if (op->bwd_chunk != 0 && (op->bwd_chunk < 32 || op->bwd_chunk > 512 || op->bwd_chunk % 2 != 0))
    return fail(c, HZ_ERR_ARG, "bwd_chunk must be 0 or even in [32, 512]");
  if (op->factor_group < 0) return fail(c, HZ_ERR_ARG, "factor_group must be >= 0");
  if (op->krylov != HZ_KRYLOV_PSEUDO_BLOCK && op->krylov != HZ_KRYLOV_BLOCK)
    return fail(c, HZ_ERR_ARG, "krylov must be HZ_KRYLOV_PSEUDO_BLOCK or HZ_KRYLOV_BLOCK");
  if (op->krylov == HZ_KRYLOV_BLOCK && op->block_size < 2)
    return fail(c, HZ_ERR_ARG, "block FGMRES needs block_size >= 2");
  const int64_t nv = md->nv, ne = md->ne, nf = md->nf;
  for (int64_t q = 0; q < ne * 4; q++)
    if (md->tets[q] < 0 || md->tets[q] >= nv) return fail(c, HZ_ERR_ARG, "tet vertex id out of range");
  for (int64_t q = 0; q < nf * 3; q++)
    if (md->faces[q] < 0 || md->faces[q] >= nv) return fail(c, HZ_ERR_ARG, "face vertex id out of range");
  P.mesh.nv = nv;
  P.mesh.ne = ne;
  P.mesh.xyz.assign(md->xyz, md->xyz + 3 * nv);
  P.mesh.tets.assign(md->tets, md->tets + 4 * ne);
  P.mesh.faces.assign(md->faces, md->faces + 3 * nf);
  P.mesh.tag.assign(md->face_tag, md->face_tag + nf);
  P.mesh.c.resize(ne);
  for (int64_t e = 0; e < ne; e++) {
    P.mesh.c[e] = cplx(md->c_re[e], md->c_im[e]);
    if (P.mesh.c[e] == cplx(0.0, 0.0)) return fail(c, HZ_ERR_ARG, "zero wave speed");
  }
  std::vector<int32_t> part;
  if (op->elem_part) {
    part.assign(op->elem_part, op->elem_part + ne);
    for (int64_t e = 0; e < ne; e++)
      if (part[e] < 0 || part[e] >= op->nsub) return fail(c, HZ_ERR_ARG, "elem_part out of range");
  } else {
    hz::rcb_partition(P.mesh, op->nsub, part);
  }
  if (op->levels == 2) {
    if (!md->coarse_xyz || !md->coarse_tets || !md->fine_parent || md->coarse_nv <= 0 || md->coarse_ne <= 0)
      return fail(c, HZ_ERR_ARG, "two levels need the nested coarse mesh");
    P.cmesh.nv = md->coarse_nv;
    P.cmesh.ne = md->coarse_ne;
    P.cmesh.xyz.assign(md->coarse_xyz, md->coarse_xyz + 3 * md->coarse_nv);
    P.cmesh.tets.assign(md->coarse_tets, md->coarse_tets + 4 * md->coarse_ne);
    P.cmesh.faces.assign(md->coarse_faces, md->coarse_faces + 3 * md->coarse_nf);
    P.cmesh.tag.assign(md->coarse_face_tag, md->coarse_face_tag + md->coarse_nf);
    P.parent.assign(md->fine_parent, md->fine_parent + ne);
    for (int64_t e = 0; e < ne; e++)
      if (P.parent[e] < 0 || P.parent[e] >= md->coarse_ne) return fail(c, HZ_ERR_ARG, "fine_parent out of range");
  }
  auto tp = std::chrono::steady_clock::now();
  phase("validate + partition", tp);
  hz::build_dofs(P.mesh, md->order, P.dofs);
  phase("dofs", tp);
  hz::assemble_global(P.mesh, P.dofs, P.A);
  phase("global assembly", tp);
  hz::build_subdomains(P.mesh, P.dofs, part, op->nsub, op->overlap, P.subs);
  phase("subdomains + local A_i", tp);
  const int prec_k = op->precision == HZ_FP64 ? 112 : 128;
  int leaf = op->leaf_size > 0 ? op->leaf_size : 64;
  int maxsn = op->max_snode > 0 ? op->max_snode : 128;
  maxsn = std::min(maxsn, prec_k);
  leaf = std::max(leaf, 1);
  {
    std::vector<hz::MatrixInput> mats(op->nsub);
    std::vector<std::vector<double>> coords(op->nsub);
    for (int i = 0; i < op->nsub; i++) {
      const hz::Subdomain& S = P.subs[i];
      coords[i].resize(S.dofs.size() * 3);
      for (size_t k = 0; k < S.dofs.size(); k++)
        for (int a = 0; a < 3; a++) coords[i][3 * k + a] = P.dofs.coord[3 * S.dofs[k] + a];
      mats[i].A = &S.A;
      mats[i].coord = coords[i].data();
      mats[i].gidx = S.dofs.data();
      mats[i].weight = S.D.data();
      mats[i].release = &P.subs[i].A;     // its values live on in the symbolic entries
      P.nnz_local += S.A.pat.nnz();
    }
    hz::symbolic_batch(mats, leaf, maxsn, P.local, op->factor_group);
  }
  phase("local symbolic", tp);
  if (op->levels == 2 && op->coarse_solver == HZ_COARSE_ORAS) {
    hz::build_coarse(P, true);
    phase("coarse space", tp);
    hz::build_coarse_subdomains(P, part, op->nsub, op->overlap);
    phase("coarse subdomains + E_i", tp);
    std::vector<hz::MatrixInput> mats(op->nsub);
    std::vector<std::vector<double>> coords(op->nsub);
    for (int i = 0; i < op->nsub; i++) {
      const hz::Subdomain& S = P.csubs[i];
      coords[i].resize(S.dofs.size() * 3);
      for (size_t k = 0; k < S.dofs.size(); k++)
        for (int a = 0; a < 3; a++) coords[i][3 * k + a] = P.cdofs.coord[3 * S.dofs[k] + a];
      mats[i].A = &S.A;
      mats[i].coord = coords[i].data();
      mats[i].gidx = P.cgidx[i].data();
      mats[i].weight = S.D.data();
      mats[i].release = &P.csubs[i].A;
    }
    hz::symbolic_batch(mats, leaf, maxsn, P.clocal, op->factor_group);
    phase("coarse local symbolic", tp);
  } else if (op->levels == 2) {
    hz::build_coarse(P);
    std::vector<double> coords(P.nH * 3);
    std::vector<int64_t> gid(P.nH);
    std::vector<double> one(P.nH, 1.0);
    for (int64_t k = 0; k < P.cdofs.n; k++)
      if (P.cfree[k] >= 0)
        for (int a = 0; a < 3; a++) coords[3 * P.cfree[k] + a] = P.cdofs.coord[3 * k + a];
    for (int64_t k = 0; k < P.nH; k++) gid[k] = k;
    hz::MatrixInput mi{&P.E, coords.data(), gid.data(), one.data()};
    phase("coarse space", tp);
    hz::symbolic_batch({mi}, leaf, 112, P.coarse);
    phase("coarse symbolic", tp);
  }
  return HZ_OK;
}

static void fill_stats(hz_ctx* c, const hz::HostProblem& P) {
  hz_stats& s = c->stats;
  s.n = P.dofs.n;
  s.nnz = P.A.pat.nnz();
  s.n_coarse = P.nH;
  s.nnz_coarse = P.E.pat.nnz();
  s.sum_ni = P.local.voff.empty() ? 0 : P.local.voff.back();
  s.nnz_local = P.nnz_local;
  s.nnz_factor = P.local.panel_elems;
  const bool it = !P.clocal.voff.empty();           // iterative coarse solve
  s.nnz_factor_coarse = it ? P.clocal.panel_elems : P.coarse.panel_elems;
  s.nsupernodes = int64_t(P.local.sn_k.size());
  s.nlevels = P.local.nlev;
  s.nlevels_coarse = it ? P.clocal.nlev : P.coarse.nlev;
  const int64_t vs = c->opt.precision == HZ_FP64 ? 16 : 8;
  s.front_bytes = std::max({P.local.front_elems * vs, P.coarse.front_elems * 16, P.clocal.front_elems * vs});
  s.factor_flops = P.local.flops;
  s.coarse_solve_levels = s.nlevels_coarse;
  s.coarse_merged_chains = 0;
  s.coarse_merged_bytes = 0;
  {
    const int prec = c->opt.precision == HZ_MIXED ? 1 : 0;
    const SolveTree T = plan_solve_tree(P.local, local_merge_width(prec), local_merge_sparse(P.local));
    s.solve_levels = T.nlev;
    s.merged_chains = 0;
    for (const auto& ch : T.chains) s.merged_chains += ch.size() > 1;
    s.merged_bytes = T.merged_elems * vs;
  }
  if (!it && !P.coarse.voff.empty()) {
    const SolveTree T = plan_solve_tree(P.coarse, hz::kMaxSolveK);
    s.coarse_solve_levels = T.nlev;
    for (const auto& ch : T.chains) s.coarse_merged_chains += ch.size() > 1;
    s.coarse_merged_bytes = T.merged_elems * 16;
  }
}

extern "C" hz_status hz_plan(const hz_mesh_desc* md, const hz_options* op, hz_stats* out) {
  if (!out) return HZ_ERR_ARG;
  hz_ctx tmp;
  if (op) tmp.opt = *op;
  auto t0 = std::chrono::steady_clock::now();
  hz::HostProblem P;
  hz_status s = analyse(&tmp, md, op, P);
  if (s != HZ_OK) {
    std::fprintf(stderr, "hz_plan: %s\n", tmp.err.c_str());
    return s;
  }
  fill_stats(&tmp, P);
  {
    const int prec = op->precision == HZ_MIXED ? 1 : 0;
    const int rows = op->bwd_chunk > 0 ? op->bwd_chunk : (prec == 1 ? 512 : 256);
    const SolveTree T = plan_solve_tree(P.local, local_merge_width(prec), local_merge_sparse(P.local));
    const SweepPlan sp = plan_sweeps(T.view(), prec, rows, op->sweep_tasks);     // the sweeps' tree
    const SweepPlan spf = plan_sweeps(view_of(P.local), prec, rows, op->sweep_tasks);   // the factor's
    hz_stats& st = tmp.stats;
    st.fwd_levels_wide = sp.fwd_wide;
    st.fwd_levels_narrow = sp.fwd_narrow;
    st.bwd_levels_wide = sp.bwd_wide;
    st.bwd_levels_narrow = sp.bwd_narrow;
    st.bwd_split_blocks = sp.bwd_split;
    st.tc_tiles = spf.tc_tiles;
    st.tc_multi_fronts = spf.tc_multi;
    st.tc_max_kstages = spf.tc_kstages;
    st.max_snode_width = spf.max_k;
  }
  tmp.stats.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // device bytes a context would hold after hz_factor (excluding transient fronts)
  int64_t persistent = 0, transient = 0;
  hz_engine::plan_bytes(P, *op, persistent, transient);
  tmp.stats.device_bytes = persistent;
  *out = tmp.stats;
  return HZ_OK;
}

// Device side of a context from an analysed problem: operator, interpolation, factor
// stores and Krylov workspaces.  The problem is left intact when copy_mesh is set
// (a cached analysis reused by the serving layer), else its mesh is moved out.
static hz_status populate(hz_ctx* c, hz::HostProblem& P, int order, const hz_options* op, bool copy_mesh) {
  c->st = reinterpret_cast<cudaStream_t>(op->stream);
  c->order = order;
  c->levels = op->levels;
  c->restart = op->restart;
  c->precision = op->precision;
  c->max_iter = op->max_iter > 0 ? op->max_iter : 1000;
  c->n = P.dofs.n;
  c->nnz = P.A.pat.nnz();
  c->nH = P.nH;
  c->nnzH = P.E.pat.nnz();
  c->zeta_nnz = P.Z.nnz();
  fill_stats(c, P);
#define SETUP_TRY(expr)                      \
  do {                                       \
    hz_status s_ = (expr);                   \
    if (s_ != HZ_OK) return s_;              \
  } while (0)
  SETUP_TRY(upload(c, &c->d_rp, P.A.pat.ptr));
  SETUP_TRY(upload(c, &c->d_ci, P.A.pat.col));
  SETUP_TRY(upload(c, &c->d_K, P.A.K));
  SETUP_TRY(upload(c, &c->d_M, to_d2(P.A.M)));
  SETUP_TRY(upload(c, &c->d_B, to_d2(P.A.B)));
  SETUP_TRY(dalloc(c, &c->d_A, c->nnz));
  // backward row chunks: long ones where the sweep streams complex64 panels from HBM,
  // short ones where it is limited by FP64 arithmetic (more CTAs per supernode)
  {
    const int bs = op->block_size;
    c->S = bs <= 1 ? 0 : (bs <= 4 ? 4 : (bs <= 8 ? 8 : 16));
    if (bs > 16) {
      c->err = "block_size must be at most 16";
      return HZ_ERR_ARG;
    }
  }
  SETUP_TRY(upload_factor(c, P.local, op->precision == HZ_MIXED ? 1 : 0, c->n, c->loc, c->loc_max,
                          op->precision == HZ_MIXED ? 512 : 256, c->S, op->sweep_tasks, op->bwd_chunk,
                          local_merge_width(op->precision == HZ_MIXED ? 1 : 0), local_merge_sparse(P.local)));
  {
    const hz::FactorDev& F = c->loc;
    hz_stats& st = c->stats;
    st.fwd_levels_wide = F.v_fwd_wide;
    st.fwd_levels_narrow = F.v_fwd_narrow;
    st.bwd_levels_wide = F.v_bwd_wide;
    st.bwd_levels_narrow = F.v_bwd_narrow;
    st.bwd_split_blocks = F.v_bwd_split;
    st.tc_tiles = F.v_tc_tiles;
    st.tc_multi_fronts = F.v_tc_multi;
    st.tc_max_kstages = F.v_tc_kstages;
    st.max_snode_width = F.v_max_k;
  }
  const int tc_wait = op->tc_wait_limit == 0 ? (1 << 22) : std::max(op->tc_wait_limit, 0);
  c->loc.tc_wait = tc_wait;
  if (c->levels == 2) {
    SETUP_TRY(upload(c, &c->d_Zrp, P.Z.ptr));
    SETUP_TRY(upload(c, &c->d_Zci, P.Z.col));
    SETUP_TRY(upload(c, &c->d_Zv, P.Zv));
    SETUP_TRY(upload(c, &c->d_Ztrp, P.Zt.ptr));
    SETUP_TRY(upload(c, &c->d_Ztci, P.Zt.col));
    SETUP_TRY(upload(c, &c->d_Ztv, P.Ztv));
    if (op->coarse_solver == HZ_COARSE_ORAS) {
      c->coarse_oras = 1;
      c->cmaxit = op->coarse_maxit > 0 ? op->coarse_maxit : 30;
      c->ctol = op->coarse_tol > 0.0 ? op->coarse_tol : 1e-2;
      SETUP_TRY(upload_factor(c, P.clocal, op->precision == HZ_MIXED ? 1 : 0, c->nH, c->cloc, c->cloc_max,
                              op->precision == HZ_MIXED ? 512 : 256, 0, op->sweep_tasks, op->bwd_chunk));
      c->cloc.tc_wait = tc_wait;
      SETUP_TRY(upload(c, &c->d_Erp, P.E.pat.ptr));
      SETUP_TRY(upload(c, &c->d_Eci, P.E.pat.col));
      SETUP_TRY(upload(c, &c->d_EK, P.E.K));
      SETUP_TRY(upload(c, &c->d_EM, to_d2(P.E.M)));
      SETUP_TRY(upload(c, &c->d_EB, to_d2(P.E.B)));
      SETUP_TRY(dalloc(c, &c->d_E, c->nnzH));
      const int mH = c->cmaxit;
      SETUP_TRY(dalloc(c, &c->VH, c->nH * (mH + 1)));
      SETUP_TRY(dalloc(c, &c->ZH, c->nH * mH));
      SETUP_TRY(dalloc(c, &c->wH, c->nH));
      SETUP_TRY(dalloc(c, &c->HH, int64_t(mH + 1) * mH));
      SETUP_TRY(dalloc(c, &c->snH, mH));
      SETUP_TRY(dalloc(c, &c->gH, mH + 1));
      SETUP_TRY(dalloc(c, &c->yHs, mH));
      SETUP_TRY(dalloc(c, &c->csH, mH));
      SETUP_TRY(dalloc(c, &c->scalH, 8));
      SETUP_TRY(dalloc(c, &c->brkH, 1));
    } else {
      SETUP_TRY(upload_factor(c, P.coarse, 0, c->nH, c->crs, c->crs_max, 256, c->S, op->sweep_tasks,
                              op->bwd_chunk, hz::kMaxSolveK));
    }
    SETUP_TRY(dalloc(c, &c->rH, c->nH));
    SETUP_TRY(dalloc(c, &c->yH, c->nH));
  }
  const int64_t n = c->n;
  const int m = c->restart;
  c->rk = op->recycle;
  if (c->rk > 0) {
    // [C (rk columns, right-aligned), V (m + 1 columns)] in one block; recycled-space buffers
    SETUP_TRY(dalloc(c, &c->Vx, n * (c->rk + m + 1)));
    c->V = c->Vx + int64_t(c->rk) * n;
    SETUP_TRY(dalloc(c, &c->Ux, n * c->rk));
    SETUP_TRY(dalloc(c, &c->Uh, n * c->rk));
    SETUP_TRY(dalloc(c, &c->Uxt, n * c->rk));
    SETUP_TRY(dalloc(c, &c->Uht, n * c->rk));
    SETUP_TRY(dalloc(c, &c->Ctmp, n * c->rk));
    SETUP_TRY(dalloc(c, &c->Hraw, int64_t(m + 1) * m));
    SETUP_TRY(dalloc(c, &c->Braw, int64_t(c->rk) * m));
    SETUP_TRY(dalloc(c, &c->dcoef, int64_t(hz::kComboMaxCols) * hz::kComboMaxOut));
  } else {
    SETUP_TRY(dalloc(c, &c->V, n * (m + 1)));
  }
  SETUP_TRY(dalloc(c, &c->Zs, n * m));
  SETUP_TRY(dalloc(c, &c->w, n));
  SETUP_TRY(dalloc(c, &c->b, n));
  SETUP_TRY(dalloc(c, &c->x, n));
  SETUP_TRY(dalloc(c, &c->y, n));
  SETUP_TRY(dalloc(c, &c->t, n));
  SETUP_TRY(dalloc(c, &c->partial, int64_t(hz::cgs_blocks()) * 65));
  SETUP_TRY(dalloc(c, &c->h1, 65));
  SETUP_TRY(dalloc(c, &c->h2, 65));
  SETUP_TRY(dalloc(c, &c->nrm, 65));
  SETUP_TRY(dalloc(c, &c->H, int64_t(m + 1) * m));
  SETUP_TRY(dalloc(c, &c->sn, m));
  SETUP_TRY(dalloc(c, &c->g, m + 1));
  SETUP_TRY(dalloc(c, &c->ysol, m));
  SETUP_TRY(dalloc(c, &c->cs, m));
  SETUP_TRY(dalloc(c, &c->scal, 8));
  c->gexec.assign(size_t(m) * size_t(c->rk + 1), nullptr);
  c->gcount.assign(size_t(m) * size_t(c->rk + 1), 0);
  // the iterative coarse solve waits on the host inside each preconditioner application
  c->graphs = std::getenv("HZ_NO_GRAPHS") == nullptr && !c->coarse_oras;
  SETUP_TRY(dalloc(c, &c->brk, 1));
  SETUP_TRY(dalloc(c, &c->status, 1));
  if (c->S) {
    const int S = c->S;
    // block GCRO-DR keeps its recycled space C in the rk columns right before Vb
    const int64_t vb_extra = op->krylov == HZ_KRYLOV_BLOCK ? c->rk : 0;
    SETUP_TRY(dalloc(c, &c->Vb, int64_t(S) * n * (m + 1) + vb_extra * n));
    if (c->Vb) c->Vb += vb_extra * n;
    SETUP_TRY(dalloc(c, &c->Zb, int64_t(S) * n * m));
    SETUP_TRY(dalloc(c, &c->Wc, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->Bc, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->Xc, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->Xi, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->Yi, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->Ti, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->Wi, int64_t(S) * n));
    SETUP_TRY(dalloc(c, &c->yi, int64_t(S) * n));
    if (c->levels == 2) {
      SETUP_TRY(dalloc(c, &c->rHi, int64_t(S) * c->nH));
      SETUP_TRY(dalloc(c, &c->yHi, int64_t(S) * c->nH));
    }
    SETUP_TRY(dalloc(c, &c->Hb, int64_t(S) * (m + 1) * m));
    SETUP_TRY(dalloc(c, &c->snb, int64_t(S) * m));
    SETUP_TRY(dalloc(c, &c->gb, int64_t(S) * (m + 1)));
    SETUP_TRY(dalloc(c, &c->yb, int64_t(S) * m));
    SETUP_TRY(dalloc(c, &c->csb, int64_t(S) * m));
    SETUP_TRY(dalloc(c, &c->scalb, int64_t(S) * 8));
    SETUP_TRY(dalloc(c, &c->brkb, int64_t(S)));
    SETUP_TRY(dalloc(c, &c->partial_s, int64_t(S) * hz::cgs_blocks() * 65));
    SETUP_TRY(dalloc(c, &c->h1s, int64_t(S) * 65));
    SETUP_TRY(dalloc(c, &c->h2s, int64_t(S) * 65));
    SETUP_TRY(dalloc(c, &c->nrms, int64_t(S) * 65));
    c->slots.assign(S, hz_ctx::Slot{});
    c->krylov = op->krylov;
    if (c->krylov == HZ_KRYLOV_BLOCK) {
      const int64_t nch = (int64_t(m) * S + c->rk + 63) / 64;
      SETUP_TRY(dalloc(c, &c->hblk, 2 * nch * S * 65));
      SETUP_TRY(dalloc(c, &c->yblk, int64_t(m) * S * S));
    }
  }
  // pinned scalars: 8 for the single-RHS loop, then 16 x 8 per-RHS scalars and 16 flags
  if (cudaMallocHost((void**)&c->h_pin, hz_ctx::PIN_TOTAL * sizeof(double)) != cudaSuccess) {
    c->err = "cudaMallocHost failed";
    return HZ_ERR_CUDA;
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) {
    c->err = "stream sync after upload failed";
    return HZ_ERR_CUDA;
  }
  if (copy_mesh) {
    c->mesh = P.mesh;
    c->dofs = P.dofs;
  } else {
    c->mesh = std::move(P.mesh);
    c->dofs = std::move(P.dofs);
  }
  return HZ_OK;
#undef SETUP_TRY
}

extern "C" hz_status hz_setup_mesh(const hz_mesh_desc* md, const hz_options* op, hz_ctx** outp) {
  if (!outp) return HZ_ERR_ARG;
  *outp = nullptr;
  hz_ctx* c = new hz_ctx();
  if (op) c->opt = *op;
  auto t0 = std::chrono::steady_clock::now();
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
      std::fprintf(stderr, "hz_setup_mesh: no CUDA device: %s\n", cudaGetErrorString(e));
      delete c;
      return HZ_ERR_CUDA;
    }
    c->device = dev;
  }
  hz::HostProblem P;
  hz_status s = analyse(c, md, op, P);
  if (s == HZ_OK) s = populate(c, P, md->order, op, false);
  if (s != HZ_OK) {
    std::fprintf(stderr, "hz_setup_mesh: %s\n", c->err.c_str());
    hz_free(c);
    return s;
  }
  c->stats.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *outp = c;
  return HZ_OK;
}

extern "C" hz_status hz_factor(hz_ctx* c, double freq_hz) {
  TRY(check_ctx(c));
  if (!(freq_hz > 0.0) || !std::isfinite(freq_hz)) return fail(c, HZ_ERR_ARG, "frequency must be positive");
  auto t0 = std::chrono::steady_clock::now();
  c->factored = false;
  const double w = 2.0 * M_PI * freq_hz;
  hz::launch_fill_values(c->nnz, c->d_K, c->d_M, c->d_B, w, c->d_A, c->st);
  if (c->spmv_lanes == 0) {
    const int fixed = c->opt.spmv_lanes;
    if (fixed == 2 || fixed == 4 || fixed == 8 || fixed == 16)
      c->spmv_lanes = fixed;
    else
      TRY(tune_spmv(c));
  }
  hz::set_spmv_lanes(c->spmv_lanes);
  double minp = 1e300;
  TRY(factor_one(c, c->loc, w, c->loc_max, minp));
  const bool tune = c->opt.tune_sweeps && !c->sweeps_tuned && c->opt.sweep_tasks == 0 && c->opt.bwd_chunk == 0;
  if (tune) {
    TRY(tune_sweeps(c, c->loc));
    hz_stats& st = c->stats;
    st.fwd_levels_wide = c->loc.v_fwd_wide;
    st.fwd_levels_narrow = c->loc.v_fwd_narrow;
    st.bwd_levels_wide = c->loc.v_bwd_wide;
    st.bwd_levels_narrow = c->loc.v_bwd_narrow;
    st.bwd_split_blocks = c->loc.v_bwd_split;
  }
  c->stats.sweep_chunk = c->loc.sweep_chunk;
  c->stats.sweep_scale = c->loc.sweep_scale;
  if (c->levels == 2 && c->coarse_oras) {
    hz::launch_fill_values(c->nnzH, c->d_EK, c->d_EM, c->d_EB, w, c->d_E, c->st);
    TRY(factor_one(c, c->cloc, w, c->cloc_max, minp));
    c->stats.coarse_solves = c->stats.coarse_iterations = 0;
  } else if (c->levels == 2) {
    TRY(factor_one(c, c->crs, w, c->crs_max, minp));
    if (tune) TRY(tune_sweeps(c, c->crs));
  }
  if (tune) c->sweeps_tuned = true;
  CU(cudaStreamSynchronize(c->st));
  c->stats.min_pivot = minp;
  if (c->opt.recycle_keep && c->rdim > 0)
    c->recycle_stale = true;                // re-based on the new operator at the next solve
  else
    c->rdim = 0;                            // a recycled space belongs to one operator
  c->stats.factor_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  c->factored = true;
  return HZ_OK;
}

extern "C" hz_status hz_apply_A(hz_ctx* c, const void* x, void* y) {
  TRY(check_ctx(c));
  if (c->spmv_lanes) hz::set_spmv_lanes(c->spmv_lanes);
  if (!x || !y) return fail(c, HZ_ERR_ARG, "null vector");
  if (!c->factored) return fail(c, HZ_ERR_STATE, "hz_factor must run first (A depends on the frequency)");
  hz::launch_spmv(c->n, c->d_rp, c->d_ci, c->d_A, (const double2*)x, nullptr, (double2*)y, c->st);
  CU(cudaGetLastError());
  return HZ_OK;
}

extern "C" hz_status hz_apply_M(hz_ctx* c, const void* v, void* z) {
  TRY(check_ctx(c));
  if (c->spmv_lanes) hz::set_spmv_lanes(c->spmv_lanes);
  if (!v || !z) return fail(c, HZ_ERR_ARG, "null vector");
  if (!c->factored) return fail(c, HZ_ERR_STATE, "hz_factor must run first");
  apply_prec(c, (const double2*)v, (double2*)z);
  CU(cudaGetLastError());
  return HZ_OK;
}

extern "C" hz_status hz_solve(hz_ctx* c, const void* rhs, int32_t nrhs, double tol, void* x, int32_t on_device,
                              hz_rhs_info* info) {
  TRY(check_ctx(c));
  if (c->spmv_lanes) hz::set_spmv_lanes(c->spmv_lanes);
  if (!rhs || !x || nrhs < 0 || !(tol > 0.0)) return fail(c, HZ_ERR_ARG, "bad solve arguments");
  if (!c->factored) return fail(c, HZ_ERR_STATE, "hz_factor must run before hz_solve");
  const int64_t n = c->n;
  hz_status worst = HZ_OK;
  if (c->S && c->krylov == HZ_KRYLOV_BLOCK && (nrhs > 1 || c->rk > 0)) {
    TRY(solve_block(c, (const double2*)rhs, nrhs, tol, (double2*)x, on_device != 0, info, worst));
    CU(cudaStreamSynchronize(c->st));
    return worst;
  }
  if (c->S && nrhs > 1) {
    TRY(solve_slots(c, (const double2*)rhs, nrhs, tol, (double2*)x, on_device != 0, info, worst));
    CU(cudaStreamSynchronize(c->st));
    return worst;
  }
  for (int32_t j = 0; j < nrhs; j++) {
    const double2* bj = (const double2*)rhs + int64_t(j) * n;
    double2* xj = (double2*)x + int64_t(j) * n;
    CU(cudaMemcpyAsync(c->b, bj, size_t(n) * 16, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->st));
    hz_rhs_info inf{};
    TRY(c->rk ? gcrodr_one(c, tol, &inf) : fgmres_one(c, tol, &inf));
    CU(cudaMemcpyAsync(xj, c->x, size_t(n) * 16, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->st));
    if (info) info[j] = inf;
    if (inf.status != HZ_OK && worst == HZ_OK) worst = hz_status(inf.status);
  }
  CU(cudaStreamSynchronize(c->st));
  return worst;
}

extern "C" hz_status hz_point_sources(hz_ctx* c, const double* xyz, int32_t nsrc, void* rhs_out, int32_t on_device) {
  if (!c || !xyz || !rhs_out || nsrc < 0) return fail(c, HZ_ERR_ARG, "bad point-source arguments");
  const int64_t n = c->n;
  std::vector<double2> B(size_t(n) * nsrc, make_double2(0.0, 0.0));
  const int nb = c->dofs.nb;
  for (int j = 0; j < nsrc; j++) {
    int64_t e = -1;
    double lam[4], phi[10];
    if (!hz::locate_point(c->mesh, xyz + 3 * j, e, lam)) return fail(c, HZ_ERR_ARG, "source outside the mesh");
    hz::eval_basis(c->order, lam, phi);
    for (int a = 0; a < nb; a++) {
      const int64_t g = c->dofs.elem[int64_t(nb) * e + a];
      if (!c->dofs.is_dir[g]) B[size_t(j) * n + g].x -= phi[a];
    }
  }
  if (on_device) {
    TRY(check_ctx(c));
    CU(cudaMemcpyAsync(rhs_out, B.data(), B.size() * 16, cudaMemcpyHostToDevice, c->st));
    CU(cudaStreamSynchronize(c->st));
  } else {
    std::memcpy(rhs_out, B.data(), B.size() * 16);
  }
  return HZ_OK;
}

extern "C" hz_status hz_profile(hz_ctx* c, int32_t reps, hz_profile_out* out) {
  TRY(check_ctx(c));
  if (c->spmv_lanes) hz::set_spmv_lanes(c->spmv_lanes);
  if (!out || reps < 1) return fail(c, HZ_ERR_ARG, "bad profile arguments");
  if (!c->factored) return fail(c, HZ_ERR_STATE, "hz_factor must run first");
  std::memset(out, 0, sizeof(*out));
  const int64_t n = c->n;
  const int m = c->restart;
  const int jj = std::max(1, m / 2);
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  // finite, normal test data in the vectors and the Krylov basis
  CU(cudaMemsetAsync(c->V, 0x3f, size_t(n) * (m + 1) * 16, st));
  CU(cudaMemsetAsync(c->w, 0x3f, size_t(n) * 16, st));
  CU(cudaMemsetAsync(c->b, 0x3f, size_t(n) * 16, st));
  hz::launch_cgs(n, 0, c->V, n, nullptr, c->b, 0, c->partial, st);
  hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
  hz::launch_init_cycle(c->nrm, c->g, m, c->scal + 2, c->scal + 3, st);
  c->h_pin[6] = 1.0;
  CU(cudaMemcpyAsync(c->scal + 4, c->h_pin + 6, sizeof(double), cudaMemcpyHostToDevice, st));
  const double nt = 16.0;
  auto run = [&](int ph) {
    switch (ph) {
      case HZ_PH_SPMV: hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, c->b, nullptr, c->w, st); break;
      case HZ_PH_COARSE:
        if (c->levels == 2) {
          hz::launch_spmv_real(c->nH, c->d_Ztrp, c->d_Ztci, c->d_Ztv, c->b, c->rH, st);
          coarse_solve(c, c->rH, c->yH);
          hz::launch_spmv_real(n, c->d_Zrp, c->d_Zci, c->d_Zv, c->yH, c->y, st);
        }
        break;
      case HZ_PH_RESTRICT: hz::launch_gather(c->loc, c->b, st); break;
      case HZ_PH_LOCAL_SOLVE: hz::launch_solve(c->loc, st); break;
      case HZ_PH_PROLONG: hz::launch_prolong(c->loc, c->levels == 2 ? c->y : nullptr, c->t, st); break;
      case HZ_PH_CGS2:
        hz::launch_cgs(n, jj + 1, c->V, n, nullptr, c->w, jj + 1, c->partial, st);
        hz::launch_reduce(c->partial, nb, jj + 1, c->h1, st);
        hz::launch_cgs(n, jj + 1, c->V, n, c->h1, c->w, jj + 1, c->partial, st);
        hz::launch_reduce(c->partial, nb, jj + 1, c->h2, st);
        hz::launch_cgs(n, jj + 1, c->V, n, c->h2, c->w, 0, c->partial, st);
        hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
        break;
      case HZ_PH_PRECOND: apply_prec(c, c->b, c->t); break;
      case HZ_PH_ITERATION: {
        double2* zj = c->Zs + int64_t(jj) * n;
        apply_prec(c, c->V + int64_t(jj) * n, zj);
        hz::launch_spmv(n, c->d_rp, c->d_ci, c->d_A, zj, nullptr, c->w, st);
        hz::launch_cgs(n, jj + 1, c->V, n, nullptr, c->w, jj + 1, c->partial, st);
        hz::launch_reduce(c->partial, nb, jj + 1, c->h1, st);
        hz::launch_cgs(n, jj + 1, c->V, n, c->h1, c->w, jj + 1, c->partial, st);
        hz::launch_reduce(c->partial, nb, jj + 1, c->h2, st);
        hz::launch_cgs(n, jj + 1, c->V, n, c->h2, c->w, 0, c->partial, st);
        hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
        hz::launch_givens(0, m, c->H, c->cs, c->sn, c->g, c->h1, c->h2, c->nrm, c->scal + 4, c->scal, c->brk,
                          c->scal + 1, st);
        hz::launch_scale(n, c->w, c->scal + 1, c->V + int64_t(jj + 1) * n, st);
        break;
      }
    }
  };
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  double inner_its = 0;          // iterative coarse solve: mean inner iterations per run
  for (int ph = 0; ph < HZ_PH_COUNT; ph++) {
    run(ph);   // warm-up
    // Each phase is timed as the solve runs it: captured once as a CUDA graph and replayed
    // (eagerly where the stream cannot be captured or the phase waits on the host).
    const bool host_waits = c->coarse_oras && (ph == HZ_PH_COARSE || ph == HZ_PH_PRECOND || ph == HZ_PH_ITERATION);
    cudaGraphExec_t ge = nullptr;
    long long per_run = 0;
    if (c->graphs && st != nullptr && !host_waits) {
      const long long l0 = hz::launch_count();
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        run(ph);
        if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) {
          if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
          cudaGraphDestroy(g);
        }
      }
      cudaGetLastError();
      per_run = hz::launch_count() - l0;
      hz::add_launches(-per_run);
    }
    const long long l0 = hz::launch_count();
    const int64_t c0 = c->stats.coarse_iterations;
    if (ge) CU(cudaGraphLaunch(ge, st));                                      // warm replay
    CU(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; r++) {
      if (ge) {
        CU(cudaGraphLaunch(ge, st));
        hz::add_launches(per_run);
      } else {
        run(ph);
      }
    }
    CU(cudaEventRecord(e1, st));
    CU(cudaEventSynchronize(e1));
    if (ge) cudaGraphExecDestroy(ge);
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    out->ms[ph] = double(ms) / reps;
    out->launches[ph] = (hz::launch_count() - l0) / reps;
    if (ph == HZ_PH_COARSE) inner_its = double(c->stats.coarse_iterations - c0) / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(cudaGetLastError());
  if (const char* vb = std::getenv("HZ_VERBOSE"); vb && std::atoi(vb) >= 2) {
    // diagnostics: live time of every tree level of the local and coarse sweeps (one run)
    for (hz::FactorDev* Fp : {&c->loc, &c->crs}) {
      hz::FactorDev& F = *Fp;
      if (F.nsn == 0) continue;
      const char* name = Fp == &c->loc ? "local" : "coarse";
      std::vector<cudaEvent_t> ev(size_t(2 * F.snlev + 1));
      for (auto& e : ev) cudaEventCreate(&e);
      F.level_events = ev.data();
      hz::launch_solve(F, st);
      F.level_events = nullptr;
      cudaStreamSynchronize(st);
      for (int q = 0; q < 2 * F.snlev; q++) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[size_t(q)], ev[size_t(q) + 1]);
        const bool fw = q < F.snlev;
        const int l = fw ? q : 2 * F.snlev - 1 - q;
        const int64_t nt = fw ? F.h_fwd_ptr[l + 1] - F.h_fwd_ptr[l] : F.h_bwd_ptr[l + 1] - F.h_bwd_ptr[l];
        std::fprintf(stderr, "[hz] %s %s level %3d: %6lld tasks %9.1f us\n", name, fw ? "fwd" : "bwd", l,
                     (long long)nt, 1e3 * ms);
      }
      for (auto& e : ev) cudaEventDestroy(e);
    }
  }
  // algorithmic bytes and flops
  const double nnz = double(c->nnz), dn = double(n);
  out->bytes[HZ_PH_SPMV] = nnz * (nt + 4) + (dn + 1) * 8 + 2 * dn * nt;
  out->flops[HZ_PH_SPMV] = 8 * nnz;
  if (c->levels == 2) {
    const double nz = double(c->zeta_nnz), nH = double(c->nH);
    out->bytes[HZ_PH_COARSE] = 2 * nz * 12 + (dn + 1) * 8 + (nH + 1) * 8 + 2 * dn * nt + 2 * nH * nt;
    out->flops[HZ_PH_COARSE] = 2 * 4 * nz;
    if (c->coarse_oras) {
      // per inner iteration: local coarse sweeps, E z, CGS2 at the mean position
      const double nzE = double(c->nnzH), jm = 0.5 * (inner_its + 1.0);
      const double bi = c->cloc.gather_bytes + c->cloc.solve_bytes + c->cloc.prolong_bytes +
                        nzE * (nt + 4) + (nH + 1) * 8 + 2 * nH * nt + (3 * (jm + 1) + 5) * nH * nt;
      const double fi = c->cloc.solve_flops + 8 * nzE + (32 * (jm + 1) + 12) * nH;
      out->bytes[HZ_PH_COARSE] += inner_its * bi;
      out->flops[HZ_PH_COARSE] += inner_its * fi;
    } else {
      out->bytes[HZ_PH_COARSE] += c->crs.gather_bytes + c->crs.solve_bytes + c->crs.prolong_bytes;
      out->flops[HZ_PH_COARSE] += c->crs.solve_flops;
    }
  }
  out->bytes[HZ_PH_RESTRICT] = c->loc.gather_bytes;
  out->bytes[HZ_PH_LOCAL_SOLVE] = c->loc.solve_bytes;
  out->flops[HZ_PH_LOCAL_SOLVE] = c->loc.solve_flops;
  out->bytes[HZ_PH_PROLONG] = c->loc.prolong_bytes + (c->levels == 2 ? dn * nt : 0.0);
  out->flops[HZ_PH_PROLONG] = 4.0 * double(c->loc.prolong_nnz);
  const double nc = jj + 1;
  out->bytes[HZ_PH_CGS2] = (3 * nc + 5) * dn * nt;
  out->flops[HZ_PH_CGS2] = (32 * nc + 12) * dn;
  double pb = 0, pf = 0;
  for (int ph : {HZ_PH_COARSE, HZ_PH_RESTRICT, HZ_PH_LOCAL_SOLVE, HZ_PH_PROLONG}) {
    pb += out->bytes[ph];
    pf += out->flops[ph];
  }
  if (c->levels == 2) {
    pb += out->bytes[HZ_PH_SPMV];
    pf += out->flops[HZ_PH_SPMV];
  }
  out->bytes[HZ_PH_PRECOND] = pb;
  out->flops[HZ_PH_PRECOND] = pf;
  out->bytes[HZ_PH_ITERATION] = pb + out->bytes[HZ_PH_SPMV] + out->bytes[HZ_PH_CGS2] + 2 * dn * nt;
  out->flops[HZ_PH_ITERATION] = pf + out->flops[HZ_PH_SPMV] + out->flops[HZ_PH_CGS2];
  return HZ_OK;
}

extern "C" hz_status hz_dense_eig(int32_t n, const double* A, double* w, double* V) {
  if (n < 1 || n > 1024 || !A || !w || !V) return HZ_ERR_ARG;
  std::vector<cplx> M(size_t(n) * n), ev, vec;
  for (size_t q = 0; q < M.size(); q++) M[q] = cplx(A[2 * q], A[2 * q + 1]);
  std::string err;
  if (!hz_small::eig(n, M, ev, vec, err)) return HZ_ERR_BREAKDOWN;
  for (int i = 0; i < n; i++) {
    w[2 * i] = ev[size_t(i)].real();
    w[2 * i + 1] = ev[size_t(i)].imag();
  }
  for (size_t q = 0; q < vec.size(); q++) {
    V[2 * q] = vec[q].real();
    V[2 * q + 1] = vec[q].imag();
  }
  return HZ_OK;
}

extern "C" hz_status hz_cgs2(hz_ctx* c, const void* V, int64_t ldv, int32_t ncols, void* w, void* h, double* wnorm) {
  TRY(check_ctx(c));
  if (!V || !w || !h || !wnorm) return fail(c, HZ_ERR_ARG, "null pointer");
  if (ncols < 1 || ncols > 64) return fail(c, HZ_ERR_ARG, "ncols must be in [1, 64]");
  if (ldv < c->n) return fail(c, HZ_ERR_ARG, "ldv < n");
  const int64_t n = c->n;
  const int nb = hz::cgs_blocks();
  cudaStream_t st = c->st;
  const double2* Vd = (const double2*)V;
  double2* wd = (double2*)w;
  hz::launch_cgs(n, ncols, Vd, ldv, nullptr, wd, ncols, c->partial, st);
  hz::launch_reduce(c->partial, nb, ncols, c->h1, st);
  hz::launch_cgs(n, ncols, Vd, ldv, c->h1, wd, ncols, c->partial, st);
  hz::launch_reduce(c->partial, nb, ncols, c->h2, st);
  hz::launch_cgs(n, ncols, Vd, ldv, c->h2, wd, 0, c->partial, st);
  hz::launch_reduce(c->partial, nb, 0, c->nrm, st);
  hz::launch_add2(ncols, c->h1, c->h2, (double2*)h, st);
  CU(cudaMemcpyAsync(c->h_pin + 5, &c->nrm[64].x, sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *wnorm = std::sqrt(c->h_pin[5]);
  return HZ_OK;
}

// ---------------------------------------------------------------------------
// Internal interface for the serving layer (engine.h).
// ---------------------------------------------------------------------------
namespace hz_engine {

hz_status analyse_problem(const hz_mesh_desc* md, const hz_options* op, hz::HostProblem& P, std::string& err) {
  hz_ctx tmp;
  if (op) tmp.opt = *op;
  hz_status s = analyse(&tmp, md, op, P);
  if (s != HZ_OK) err = tmp.err;
  return s;
}

void plan_bytes(const hz::HostProblem& P, const hz_options& op, int64_t& persistent, int64_t& transient) {
  const int64_t vs = op.precision == HZ_FP64 ? 16 : 8;
  const int64_t n = P.dofs.n, m = op.restart;
  const int bs = op.block_size;
  const int64_t S = bs <= 1 ? 0 : (bs <= 4 ? 4 : (bs <= 8 ? 8 : 16));
  int64_t b = 0;
  b += P.A.pat.nnz() * (4 + 8 + 16 + 16 + 16) + (n + 1) * 8;                  // A pattern, K, M', B', A
  b += P.local.panel_elems * vs + (3 * P.local.voff.back() + P.local.u_elems) * vs;
  b += plan_solve_tree(P.local, local_merge_width(op.precision == HZ_MIXED ? 1 : 0), local_merge_sparse(P.local))
           .merged_elems * vs;                                                // merged solve panels
  b += int64_t(P.local.rowlist.size()) * 4 + int64_t(P.local.cidx.size()) * 8 + int64_t(P.local.epos.size()) * 40;
  b += P.coarse.panel_elems * 16;
  if (!P.coarse.voff.empty() && P.clocal.voff.empty())
    b += plan_solve_tree(P.coarse, hz::kMaxSolveK).merged_elems * 16;          // merged solve panels
  if (!P.coarse.voff.empty())
    b += (3 * P.coarse.voff.back() + P.coarse.u_elems) * 16 + int64_t(P.coarse.epos.size()) * 40;
  if (!P.clocal.voff.empty()) {
    const int64_t mH = op.coarse_maxit > 0 ? op.coarse_maxit : 30;
    b += P.clocal.panel_elems * vs + (3 * P.clocal.voff.back() + P.clocal.u_elems) * vs +
         int64_t(P.clocal.epos.size()) * 40;
    b += P.E.pat.nnz() * (4 + 8 + 16 + 16 + 16) + (P.nH + 1) * 8 + (2 * mH + 2) * P.nH * 16;
  }
  b += (P.Z.nnz() + P.Zt.nnz()) * 12;
  b += (2 * m + 8) * n * 16;                                                   // one-RHS Krylov
  if (S) b += S * n * (2 * m + 9) * 16 + S * (P.local.voff.back() + P.local.u_elems) * 3 * vs;
  persistent = b + b / 20 + (64 << 20);                                        // 5 % + 64 MB headroom
  const int64_t tl = std::max(P.local.front_elems, P.clocal.front_elems) * vs, tc = P.coarse.front_elems * 16;
  transient = std::max(tl, tc) + std::max(tl, tc) / 10;
}

hz_status create(const hz::HostProblem& P, int order, const hz_options* op, hz_ctx** out, std::string& err) {
  *out = nullptr;
  if (!op || op->block_size < 2) {
    err = "serving contexts need block_size >= 2";
    return HZ_ERR_ARG;
  }
  hz_ctx* c = new hz_ctx();
  c->opt = *op;
  auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    delete c;
    return HZ_ERR_CUDA;
  }
  hz_status s = populate(c, const_cast<hz::HostProblem&>(P), order, op, true);
  if (s != HZ_OK) {
    err = c->err;
    hz_free(c);
    return s;
  }
  c->stats.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return HZ_OK;
}

int64_t device_bytes(const hz_ctx* c) { return c ? c->bytes : 0; }

}  // namespace hz_engine
