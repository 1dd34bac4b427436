// Host-side data structures of the hz library (setup phase, not timed).
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace hz {

using cplx = std::complex<double>;

struct Mesh {
  int64_t nv = 0, ne = 0;
  std::vector<double> xyz;       // nv*3
  std::vector<int32_t> tets;     // ne*4
  std::vector<int32_t> faces;    // nf*3
  std::vector<int8_t> tag;       // nf
  std::vector<cplx> c;           // ne (empty for the coarse mesh)
};

// Global dof numbering: vertices, then edges sorted by (min, max) vertex.
struct Dofs {
  int order = 1, nb = 4, nbf = 3;  // dofs per tet / per face
  int64_t nv = 0, n = 0;
  std::vector<int64_t> edge_key;   // sorted (min*nv + max)
  std::vector<int64_t> elem;       // ne*nb global dofs per element
  std::vector<double> coord;       // n*3 node coordinates
  std::vector<uint8_t> is_dir;     // n
  int64_t edge_id(int64_t a, int64_t b) const;
  void face_dofs(const int32_t* f, int64_t* out) const;
};

struct Csr {
  int64_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
  int64_t find(int64_t r, int64_t c) const;  // position of (r,c) or -1
};

// Frequency-free pieces of A = K - w^2 M - i w B on one pattern (Dirichlet folded:
// K holds the identity on Dirichlet rows, M and B hold zero there).
struct Parts {
  Csr pat;
  std::vector<double> K;
  std::vector<cplx> M, B;
};

struct Subdomain {
  std::vector<int64_t> elems;      // Gamma_i elements
  std::vector<int64_t> dofs;       // sorted global ids (R_i)
  std::vector<double> D;           // partition of unity on dofs
  Parts A;                         // local operator pieces in local numbering
};

// Symbolic multifrontal factorisation of a batch of sparse symmetric matrices.
struct SymbolicSet {
  int nmat = 0;
  std::vector<int64_t> voff;               // nmat+1 offsets into the concatenated vector
  std::vector<int32_t> gidx;               // voff.back(): global index of each (matrix, ND position)
  std::vector<double> weight;              // voff.back(): prolongation weight (PU or 1)
  // supernodes
  std::vector<int32_t> sn_mat, sn_k, sn_m, sn_first, sn_parent, sn_level;
  std::vector<int64_t> sn_rowoff, sn_frontoff, sn_paneloff, sn_uoff;
  std::vector<int32_t> rowlist;            // concatenated rows (vector indices), sum m
  int nlev = 0;
  std::vector<int32_t> lev_ptr, lev_sn;    // supernodes grouped by level
  // entries of the lower triangles: front position and frequency-free values
  std::vector<int64_t> epos;           // grouped by level: ent_ptr[l] .. ent_ptr[l+1]
  std::vector<int64_t> ent_ptr;
  std::vector<int64_t> ent_gptr;       // nlev * (groups + 1): entries of each (level, group)
  std::vector<double> ek;
  std::vector<cplx> em, eb;
  // extend-add: relative positions of each child's contribution rows in its parent
  std::vector<int64_t> sn_reloff;
  std::vector<int32_t> rel;
  // forward-solve contributors: for each row slot of each supernode, u-workspace indices
  std::vector<int64_t> cptr;
  std::vector<int64_t> cidx;
  int64_t front_elems = 0, panel_elems = 0, u_elems = 0;
  double flops = 0;                        // real flops of the numeric factorisation
  // factorisation groups: supernodes [grp_sn[g], grp_sn[g + 1]) (whole matrices), each
  // group's fronts planned from offset 0 of the same workspace
  std::vector<int32_t> grp_sn;
};

struct HostProblem {
  Mesh mesh, cmesh;
  std::vector<int32_t> parent;
  Dofs dofs, cdofs;
  Parts A;                            // global operator pieces
  std::vector<Subdomain> subs;
  int64_t nnz_local = 0;              // nonzeros of all A_i (their values are released after analysis)
  SymbolicSet local;                  // all A_i
  // coarse level
  int64_t nH = 0;
  std::vector<int64_t> cfree;         // coarse dof -> free index (-1 Dirichlet)
  Csr Z, Zt;                          // n x nH and nH x n
  std::vector<double> Zv, Ztv;
  Parts E;                            // coarse operator pieces
  SymbolicSet coarse;                 // direct coarse solve: LDL^T of E
  // iterative coarse solve: one-level ORAS on the coarse mesh (same partition)
  std::vector<double> cEK;            // per coarse element Galerkin pieces (transient)
  std::vector<cplx> cEM, cEB;
  std::vector<int32_t> cpart;         // coarse element -> part
  std::vector<Subdomain> csubs;       // Gamma_H,i with E_i pieces (dofs: full coarse ids)
  std::vector<std::vector<int64_t>> cgidx;   // free coarse id of each local dof (0: Dirichlet)
  SymbolicSet clocal;                 // LDL^T of all E_i
};

// setup.cpp
void build_dofs(const Mesh& m, int order, Dofs& d);
void assemble_global(const Mesh& m, const Dofs& d, Parts& A);
void rcb_partition(const Mesh& m, int nparts, std::vector<int32_t>& part);
void build_subdomains(const Mesh& m, const Dofs& d, const std::vector<int32_t>& part, int nsub,
                      int overlap, std::vector<Subdomain>& subs);
void build_coarse(HostProblem& P, bool keep_pieces = false);
void build_coarse_subdomains(HostProblem& P, const std::vector<int32_t>& part, int nsub, int overlap);
bool locate_point(const Mesh& m, const double* p, int64_t& elem, double lam[4]);
void eval_basis(int order, const double lam[4], double* out);

// symbolic.cpp
struct MatrixInput {
  const Parts* A;
  const double* coord;        // n*3
  const int64_t* gidx;        // n: global index of each local dof (for gather/scatter)
  const double* weight;       // n: prolongation weights
  Parts* release = nullptr;   // if set (== A): emptied once its entries are copied
};
// group: matrices whose fronts are planned (and factorised) together in one frontal
// workspace; groups run one after the other and reuse it.  0: all matrices at once.
void symbolic_batch(const std::vector<MatrixInput>& mats, int leaf, int maxsn, SymbolicSet& S, int group = 0);

}  // namespace hz
