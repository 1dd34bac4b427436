// Symbolic analysis of the local direct solver (the "direct solver" of the
// method's subdomain and coarse solves): geometric nested-dissection ordering,
// supernode partition, multifrontal row structures, assembly-tree levels, and
// every index map the batched device factorisation and solves need.
#include <algorithm>
#include <cmath>
#include <iterator>
#include <map>
#include <set>
#include <numeric>

#include "host.h"

namespace hz {

namespace {

struct SymOne {
  int64_t n = 0;
  std::vector<int32_t> perm, iperm;   // perm[pos] = local dof, iperm[dof] = pos
  std::vector<int32_t> first, k;      // supernode column ranges in ND positions
  std::vector<int64_t> rowoff;        // ns + 1
  std::vector<int32_t> rows;          // ND positions, each supernode's list sorted
  std::vector<int32_t> parent, level;
  // lower-triangle entries: supernode-relative front offset (row + col*m) and source entry
  std::vector<int32_t> e_sn;
  std::vector<int64_t> e_off, e_src;
};

struct NDState {
  const Csr* pat;
  const double* coord;
  int leaf, maxsn;
  std::vector<int8_t> where;
  std::vector<int32_t> order;
  std::vector<int32_t> first, k;
};

void emit(NDState& st, const std::vector<int32_t>& ids) {
  const int32_t len = int32_t(ids.size());
  if (len == 0) return;
  const int32_t start = int32_t(st.order.size());
  st.order.insert(st.order.end(), ids.begin(), ids.end());
  const int32_t nch = (len + st.maxsn - 1) / st.maxsn;
  int32_t pos = start;
  for (int32_t c = 0; c < nch; c++) {
    const int32_t sz = len / nch + (c < len % nch ? 1 : 0);
    st.first.push_back(pos);
    st.k.push_back(sz);
    pos += sz;
  }
}

void nd_rec(NDState& st, std::vector<int32_t>& S) {
  if (int(S.size()) <= st.leaf) {
    emit(st, S);
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int32_t v : S)
    for (int i = 0; i < 3; i++) {
      lo[i] = std::min(lo[i], st.coord[3 * int64_t(v) + i]);
      hi[i] = std::max(hi[i], st.coord[3 * int64_t(v) + i]);
    }
  int ax = 0;
  for (int i = 1; i < 3; i++)
    if (hi[i] - lo[i] > hi[ax] - lo[ax]) ax = i;
  const size_t mid = S.size() / 2;
  const double* cd = st.coord;
  std::nth_element(S.begin(), S.begin() + mid, S.end(), [cd, ax](int32_t a, int32_t b) {
    const double ca = cd[3 * int64_t(a) + ax], cb = cd[3 * int64_t(b) + ax];
    return ca < cb || (ca == cb && a < b);
  });
  for (size_t q = 0; q < S.size(); q++) st.where[S[q]] = q < mid ? 0 : 1;
  // one-sided vertex separators from the edge cut; keep the smaller one
  const Csr& P = *st.pat;
  std::vector<int32_t> sepL, sepR;
  for (size_t q = 0; q < S.size(); q++) {
    const int32_t v = S[q];
    const int8_t side = st.where[v];
    for (int64_t t = P.ptr[v]; t < P.ptr[v + 1]; t++) {
      const int8_t w = st.where[P.col[t]];
      if (w >= 0 && w != side) {
        (side == 0 ? sepL : sepR).push_back(v);
        break;
      }
    }
  }
  const std::vector<int32_t>& sep = sepL.size() < sepR.size() ? sepL : sepR;
  for (int32_t v : sep) st.where[v] = 2;
  std::vector<int32_t> L, R, Sep;
  for (int32_t v : S) {
    const int8_t w = st.where[v];
    (w == 0 ? L : (w == 1 ? R : Sep)).push_back(v);
  }
  for (int32_t v : S) st.where[v] = -1;
  std::vector<int32_t>().swap(S);
  if (!L.empty()) nd_rec(st, L);
  if (!R.empty()) nd_rec(st, R);
  std::sort(Sep.begin(), Sep.end());
  emit(st, Sep);
}

void analyse_one(const MatrixInput& in, int leaf, int maxsn, SymOne& S) {
  const Csr& P = in.A->pat;
  S.n = P.n;
  NDState st;
  st.pat = &P;
  st.coord = in.coord;
  st.leaf = leaf;
  st.maxsn = maxsn;
  st.where.assign(P.n, -1);
  std::vector<int32_t> all(P.n);
  std::iota(all.begin(), all.end(), 0);
  nd_rec(st, all);
  S.perm.swap(st.order);
  S.first.swap(st.first);
  S.k.swap(st.k);
  S.iperm.assign(P.n, 0);
  for (int64_t p = 0; p < P.n; p++) S.iperm[S.perm[p]] = int32_t(p);
  const int32_t ns = int32_t(S.first.size());
  std::vector<int32_t> owner(P.n);
  for (int32_t s = 0; s < ns; s++)
    for (int32_t p = S.first[s]; p < S.first[s] + S.k[s]; p++) owner[p] = s;
  std::vector<std::vector<int32_t>> children(ns);
  S.rowoff.assign(ns + 1, 0);
  S.parent.assign(ns, -1);
  S.level.assign(ns, 0);
  std::vector<int32_t> beyond;
  for (int32_t s = 0; s < ns; s++) {
    const int32_t f = S.first[s], l = f + S.k[s];
    beyond.clear();
    for (int32_t p = f; p < l; p++) {
      const int32_t v = S.perm[p];
      for (int64_t t = P.ptr[v]; t < P.ptr[v + 1]; t++) {
        const int32_t p2 = S.iperm[P.col[t]];
        if (p2 >= l) beyond.push_back(p2);
      }
    }
    int32_t lev = 0;
    for (int32_t c : children[s]) {
      for (int64_t t = S.rowoff[c] + S.k[c]; t < S.rowoff[c + 1]; t++)
        if (S.rows[t] >= l) beyond.push_back(S.rows[t]);
      lev = std::max(lev, S.level[c] + 1);
    }
    S.level[s] = lev;
    std::sort(beyond.begin(), beyond.end());
    beyond.erase(std::unique(beyond.begin(), beyond.end()), beyond.end());
    for (int32_t p = f; p < l; p++) S.rows.push_back(p);
    S.rows.insert(S.rows.end(), beyond.begin(), beyond.end());
    S.rowoff[s + 1] = int64_t(S.rows.size());
    if (!beyond.empty()) {
      S.parent[s] = owner[beyond[0]];
      children[S.parent[s]].push_back(s);
    }
  }
  // lower-triangle entries -> (supernode, row + col*m)
  for (int64_t r = 0; r < P.n; r++)
    for (int64_t t = P.ptr[r]; t < P.ptr[r + 1]; t++) {
      const int32_t pr = S.iperm[r], pc = S.iperm[P.col[t]];
      if (pr < pc) continue;
      const int32_t s = owner[pc];
      const int64_t m = S.rowoff[s + 1] - S.rowoff[s];
      const int32_t* b = S.rows.data() + S.rowoff[s];
      const int64_t row = std::lower_bound(b, b + m, pr) - b;
      S.e_sn.push_back(s);
      S.e_off.push_back(row + int64_t(pc - S.first[s]) * m);
      S.e_src.push_back(t);
    }
}

}  // namespace

void symbolic_batch(const std::vector<MatrixInput>& mats, int leaf, int maxsn, SymbolicSet& S, int group) {
  const int nmat = int(mats.size());
  std::vector<SymOne> one(nmat);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < nmat; i++) analyse_one(mats[i], leaf, maxsn, one[i]);

  S = SymbolicSet();
  S.nmat = nmat;
  S.voff.assign(nmat + 1, 0);
  for (int i = 0; i < nmat; i++) S.voff[i + 1] = S.voff[i] + one[i].n;
  const int64_t ntot = S.voff[nmat];
  S.gidx.resize(ntot);
  S.weight.resize(ntot);
  std::vector<int32_t> sn_base(nmat + 1, 0);
  for (int i = 0; i < nmat; i++) sn_base[i + 1] = sn_base[i] + int32_t(one[i].first.size());
  const int32_t ns = sn_base[nmat];
  S.sn_mat.resize(ns);
  S.sn_k.resize(ns);
  S.sn_m.resize(ns);
  S.sn_first.resize(ns);
  S.sn_parent.resize(ns);
  S.sn_level.resize(ns);
  S.sn_rowoff.assign(ns + 1, 0);
  S.sn_frontoff.assign(ns + 1, 0);
  S.sn_paneloff.assign(ns + 1, 0);
  S.sn_uoff.assign(ns + 1, 0);
  int maxlev = 0;
  for (int i = 0; i < nmat; i++) {
    const SymOne& O = one[i];
    for (int64_t p = 0; p < O.n; p++) {
      S.gidx[S.voff[i] + p] = int32_t(mats[i].gidx[O.perm[p]]);
      S.weight[S.voff[i] + p] = mats[i].weight[O.perm[p]];
    }
    for (size_t s = 0; s < O.first.size(); s++) {
      const int32_t g = sn_base[i] + int32_t(s);
      const int64_t m = O.rowoff[s + 1] - O.rowoff[s];
      S.sn_mat[g] = i;
      S.sn_k[g] = O.k[s];
      S.sn_m[g] = int32_t(m);
      S.sn_first[g] = int32_t(S.voff[i] + O.first[s]);
      S.sn_parent[g] = O.parent[s] < 0 ? -1 : sn_base[i] + O.parent[s];
      S.sn_level[g] = O.level[s];
      maxlev = std::max(maxlev, O.level[s]);
      S.sn_rowoff[g + 1] = S.sn_rowoff[g] + m;
      S.sn_paneloff[g + 1] = S.sn_paneloff[g] + m * O.k[s];
      S.sn_uoff[g + 1] = S.sn_uoff[g] + (m - O.k[s]);
      const double k = O.k[s], r = double(m) - k;
      S.flops += 8.0 * (k * k * k / 3.0 + r * k * k + r * r * k / 2.0);
    }
  }
  S.panel_elems = S.sn_paneloff[ns];
  S.u_elems = S.sn_uoff[ns];
  S.rowlist.resize(S.sn_rowoff[ns]);
  for (int i = 0; i < nmat; i++) {
    const SymOne& O = one[i];
    const int64_t base = S.sn_rowoff[sn_base[i]];
    for (size_t t = 0; t < O.rows.size(); t++) S.rowlist[base + t] = int32_t(S.voff[i] + O.rows[t]);
  }
  // levels
  S.nlev = maxlev + 1;
  S.lev_ptr.assign(S.nlev + 1, 0);
  for (int32_t g = 0; g < ns; g++) S.lev_ptr[S.sn_level[g] + 1]++;
  for (int l = 0; l < S.nlev; l++) S.lev_ptr[l + 1] += S.lev_ptr[l];
  S.lev_sn.resize(ns);
  {
    std::vector<int32_t> fill(S.lev_ptr.begin(), S.lev_ptr.end() - 1);
    for (int32_t g = 0; g < ns; g++) S.lev_sn[fill[S.sn_level[g]]++] = g;
  }
  // factorisation groups of whole matrices
  {
    const int gsz = group > 0 ? group : std::max(nmat, 1);
    S.grp_sn.clear();
    for (int i = 0; i < nmat; i += gsz) S.grp_sn.push_back(sn_base[i]);
    S.grp_sn.push_back(ns);
  }
  // Frontal workspace: a static best-fit plan per group.  The front of supernode s is
  // allocated when its level starts and released once its parent's level has
  // absorbed it (extend-add), so only the live part of the tree is resident; the
  // groups are factorised one after the other and each plans from offset 0.
  for (size_t grp = 0; grp + 1 < S.grp_sn.size(); grp++) {
    const int32_t g0 = S.grp_sn[grp], g1 = S.grp_sn[grp + 1];
    // best fit: free blocks indexed by size (for take) and by offset (to coalesce)
    std::map<int64_t, int64_t> by_off;              // offset -> size
    std::set<std::pair<int64_t, int64_t>> by_size;  // (size, offset)
    int64_t top = 0, peak = 0;
    auto erase_size = [&](int64_t sz, int64_t off) { by_size.erase({sz, off}); };
    auto take = [&](int64_t sz) {
      auto it = by_size.lower_bound({sz, int64_t(-1)});
      if (it == by_size.end()) {
        const int64_t off = top;
        top += sz;
        peak = std::max(peak, top);
        return off;
      }
      const int64_t bsz = it->first, off = it->second;
      by_size.erase(it);
      by_off.erase(off);
      if (bsz > sz) {
        by_off[off + sz] = bsz - sz;
        by_size.insert({bsz - sz, off + sz});
      }
      return off;
    };
    auto give = [&](int64_t off, int64_t sz) {
      auto nx = by_off.lower_bound(off);
      if (nx != by_off.end() && off + sz == nx->first) {
        sz += nx->second;
        erase_size(nx->second, nx->first);
        nx = by_off.erase(nx);
      }
      if (nx != by_off.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
          erase_size(pv->second, pv->first);
          off = pv->first;
          sz += pv->second;
          by_off.erase(pv);
        }
      }
      if (off + sz == top) {        // give the tail back to the unallocated end
        top = off;
        return;
      }
      by_off[off] = sz;
      by_size.insert({sz, off});
    };
    std::vector<std::vector<int32_t>> kids(ns);
    for (int32_t g = 0; g < ns; g++)
      if (S.sn_parent[g] >= 0) kids[S.sn_parent[g]].push_back(g);
    for (int l = 0; l < S.nlev; l++) {
      for (int32_t q = S.lev_ptr[l]; q < S.lev_ptr[l + 1]; q++) {
        const int32_t g = S.lev_sn[q];
        if (g < g0 || g >= g1) continue;
        S.sn_frontoff[g] = take(int64_t(S.sn_m[g]) * S.sn_m[g]);
      }
      for (int32_t q = S.lev_ptr[l]; q < S.lev_ptr[l + 1]; q++) {
        const int32_t g = S.lev_sn[q];
        if (g < g0 || g >= g1) continue;
        for (int32_t c : kids[g]) give(S.sn_frontoff[c], int64_t(S.sn_m[c]) * S.sn_m[c]);
        if (S.sn_parent[g] < 0) give(S.sn_frontoff[g], int64_t(S.sn_m[g]) * S.sn_m[g]);
      }
    }
    S.front_elems = std::max(S.front_elems, peak);
  }
  // entries, grouped by the level of the supernode owning their column
  int64_t ne = 0;
  for (int i = 0; i < nmat; i++) ne += int64_t(one[i].e_sn.size());
  S.epos.resize(ne);
  S.ek.resize(ne);
  S.em.resize(ne);
  S.eb.resize(ne);
  S.ent_ptr.assign(S.nlev + 1, 0);
  for (int i = 0; i < nmat; i++)
    for (int32_t sl : one[i].e_sn) S.ent_ptr[S.sn_level[sn_base[i] + sl] + 1]++;
  for (int l = 0; l < S.nlev; l++) S.ent_ptr[l + 1] += S.ent_ptr[l];
  {
    // per (level, group) starts: entries are filled matrix by matrix, so each level's
    // entries are ordered by matrix and hence by group
    const int G = int(S.grp_sn.size()) - 1;
    std::vector<int64_t> cnt(size_t(S.nlev) * G, 0);
    for (int i = 0; i < nmat; i++) {
      const int g = int(std::upper_bound(S.grp_sn.begin(), S.grp_sn.end(), sn_base[i]) - S.grp_sn.begin()) - 1;
      for (int32_t sl : one[i].e_sn) cnt[size_t(S.sn_level[sn_base[i] + sl]) * G + g]++;
    }
    S.ent_gptr.assign(size_t(S.nlev) * (G + 1), 0);
    for (int l = 0; l < S.nlev; l++) {
      int64_t at = S.ent_ptr[l];
      for (int g = 0; g < G; g++) {
        S.ent_gptr[size_t(l) * (G + 1) + g] = at;
        at += cnt[size_t(l) * G + g];
      }
      S.ent_gptr[size_t(l) * (G + 1) + G] = at;
    }
  }
  {
    std::vector<int64_t> fill(S.ent_ptr.begin(), S.ent_ptr.end() - 1);
    for (int i = 0; i < nmat; i++) {
      SymOne& O = one[i];
      const Parts& A = *mats[i].A;
      for (size_t t = 0; t < O.e_sn.size(); t++) {
        const int32_t g = sn_base[i] + O.e_sn[t];
        const int64_t q = fill[S.sn_level[g]]++;
        S.epos[q] = S.sn_frontoff[g] + O.e_off[t];
        S.ek[q] = A.K[O.e_src[t]];
        S.em[q] = A.M[O.e_src[t]];
        S.eb[q] = A.B[O.e_src[t]];
      }
      // the per-entry maps and (when asked) the input values are not needed any more
      std::vector<int32_t>().swap(O.e_sn);
      std::vector<int64_t>().swap(O.e_off);
      std::vector<int64_t>().swap(O.e_src);
      if (mats[i].release) *mats[i].release = Parts();
    }
  }
  // extend-add maps and forward-solve contributors
  S.sn_reloff.assign(ns + 1, 0);
  for (int32_t g = 0; g < ns; g++)
    S.sn_reloff[g + 1] = S.sn_reloff[g] + (S.sn_parent[g] >= 0 ? S.sn_m[g] - S.sn_k[g] : 0);
  S.rel.resize(S.sn_reloff[ns]);
  S.cptr.assign(S.sn_rowoff[ns] + 1, 0);
  for (int32_t g = 0; g < ns; g++) {
    const int32_t p = S.sn_parent[g];
    if (p < 0) continue;
    const int32_t* pb = S.rowlist.data() + S.sn_rowoff[p];
    const int32_t pm = S.sn_m[p];
    for (int32_t i = S.sn_k[g]; i < S.sn_m[g]; i++) {
      const int32_t r = S.rowlist[S.sn_rowoff[g] + i];
      const int32_t pos = int32_t(std::lower_bound(pb, pb + pm, r) - pb);
      S.rel[S.sn_reloff[g] + (i - S.sn_k[g])] = pos;
      S.cptr[S.sn_rowoff[p] + pos + 1]++;
    }
  }
  for (int64_t t = 0; t < S.sn_rowoff[ns]; t++) S.cptr[t + 1] += S.cptr[t];
  S.cidx.resize(S.cptr[S.sn_rowoff[ns]]);
  {
    std::vector<int64_t> fill(S.cptr.begin(), S.cptr.end() - 1);
    for (int32_t g = 0; g < ns; g++) {
      const int32_t p = S.sn_parent[g];
      if (p < 0) continue;
      for (int32_t i = S.sn_k[g]; i < S.sn_m[g]; i++) {
        const int32_t pos = S.rel[S.sn_reloff[g] + (i - S.sn_k[g])];
        S.cidx[fill[S.sn_rowoff[p] + pos]++] = S.sn_uoff[g] + (i - S.sn_k[g]);
      }
    }
  }
}

}  // namespace hz
