// Host-side symbolic analysis of the hybrid full-space system (see fsplan.h).
#include "fsplan.h"

#include <algorithm>
#include <numeric>

namespace condipm {
namespace {

int find_blk(const FsPlan& F, int I, int J) {
  auto b = F.bci.begin() + F.brp[I], e = F.bci.begin() + F.brp[I + 1];
  auto it = std::lower_bound(b, e, J);
  if (it == e || *it != J) return -1;
  return int(it - F.bci.begin());
}

}  // namespace

std::string build_fs_plan(const Plan& P, FsPlan& F) {
  const int nb = P.nb, ng = P.ng, nw = P.nw, nx = P.nx, m = P.m;
  const int n = nw + nx + m;
  const int nlim_rows = m - 1 - ng;
  if (nlim_rows < 0) return "inconsistent h rows";
  F = FsPlan();
  F.n = n;
  // ---- unknowns -> nodes (buses 0..nb-1, limit rows nb..)
  const int nnodes = nb + nlim_rows;
  std::vector<int> node(n, -1);
  for (int i = 0; i < nb; ++i) {
    if (P.th_w[i] >= 0) node[P.th_w[i]] = i;
    node[P.vm_w[i]] = i;
    if (P.g_row_P[i] >= 0) node[nw + P.g_row_P[i]] = i;
    if (P.g_row_Q[i] >= 0) node[nw + P.g_row_Q[i]] = i;
  }
  for (int k = 1; k < ng; ++k) node[P.pg_w[k]] = P.gbus[k];
  node[nw + nx + 0] = P.slack;
  for (int k = 0; k < ng; ++k) node[nw + nx + 1 + k] = P.gbus[k];
  for (int r = 1 + ng; r < m; ++r) node[nw + nx + r] = nb + (r - 1 - ng);
  for (int u = 0; u < n; ++u)
    if (node[u] < 0) return "unknown without a block";
  std::vector<std::vector<int>> members(nnodes);
  for (int u = 0; u < n; ++u) members[node[u]].push_back(u);   // ascending natural index
  std::vector<int> wt(nnodes);
  for (int v = 0; v < nnodes; ++v) {
    wt[v] = int(members[v].size());
    if (wt[v] == 0) return "empty block";
    if (wt[v] > FS_BMAX) return "block larger than FS_BMAX";
  }
  // ---- node graph
  std::vector<std::vector<int>> adj(nnodes);
  auto link = [&](int a, int b) {
    if (a == b) return;
    adj[a].push_back(b);
    adj[b].push_back(a);
  };
  for (int l = 0; l < P.nl; ++l) link(P.lf[l], P.lt[l]);
  {
    std::vector<int> cl{P.slack};
    for (int l = 0; l < P.nl; ++l) {
      if (P.lf[l] == P.slack) cl.push_back(P.lt[l]);
      if (P.lt[l] == P.slack) cl.push_back(P.lf[l]);
    }
    for (size_t a = 0; a < cl.size(); ++a)
      for (size_t b = a + 1; b < cl.size(); ++b) link(cl[a], cl[b]);
  }
  for (size_t e = 0; e < P.end_h.size(); ++e) {
    const int r = P.end_h[e];
    if (r < 0) continue;
    const int v = nb + (r - 1 - ng);
    link(v, P.end_i[e]);
    link(v, P.end_k[e]);
  }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  // ---- ordering and positions: the flow-limit rows first (their pivots are
  // then exactly -(Sigma_s^{-1} + delta_c), and each only joins two adjacent
  // buses), then the buses by minimum degree
  std::vector<int> order;
  order.reserve(nnodes);
  for (int v = nb; v < nnodes; ++v) order.push_back(v);
  {
    std::vector<std::vector<int>> badj(nb);
    for (int v = 0; v < nb; ++v)
      for (int a : adj[v])
        if (a < nb) badj[v].push_back(a);
    std::vector<int> bwt(wt.begin(), wt.begin() + nb);
    const std::vector<int> bo = min_degree_order(nb, badj, bwt);
    if (int(bo.size()) != nb) return "ordering size mismatch";
    order.insert(order.end(), bo.begin(), bo.end());
  }
  std::vector<int> blk_of_node(nnodes, -1);
  for (int I = 0; I < nnodes; ++I) blk_of_node[order[I]] = I;
  const int nblk = nnodes;
  F.nblk = nblk;
  F.bptr.assign(nblk + 1, 0);
  for (int I = 0; I < nblk; ++I) F.bptr[I + 1] = F.bptr[I] + wt[order[I]];
  F.pos.assign(n, -1);
  std::vector<int> blk(n);
  for (int I = 0; I < nblk; ++I) {
    const auto& mem = members[order[I]];
    for (size_t t = 0; t < mem.size(); ++t) {
      F.pos[mem[t]] = F.bptr[I] + int(t);
      blk[mem[t]] = I;
    }
    F.bmax = std::max(F.bmax, int(mem.size()));
  }
  auto bsz = [&](int I) { return F.bptr[I + 1] - F.bptr[I]; };
  // ---- symbolic block elimination (column structures with children merged)
  std::vector<std::vector<int>> badj(nblk);
  for (int v = 0; v < nnodes; ++v)
    for (int a : adj[v]) badj[blk_of_node[v]].push_back(blk_of_node[a]);
  std::vector<std::vector<int>> Ls(nblk), children(nblk);
  {
    std::vector<int> mark(nblk, -1);
    for (int j = 0; j < nblk; ++j) {
      std::vector<int>& s = Ls[j];
      for (int i : badj[j])
        if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
      for (int c : children[j])
        for (int i : Ls[c])
          if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
      std::sort(s.begin(), s.end());
      if (!s.empty()) children[s[0]].push_back(j);
    }
  }
  // combined rows: L part (transposed column structures), diagonal, U part
  {
    std::vector<std::vector<int>> rows(nblk);
    for (int j = 0; j < nblk; ++j)
      for (int i : Ls[j]) rows[i].push_back(j);
    F.brp.assign(nblk + 1, 0);
    for (int i = 0; i < nblk; ++i) {
      std::vector<int>& r = rows[i];
      std::sort(r.begin(), r.end());
      r.push_back(i);
      r.insert(r.end(), Ls[i].begin(), Ls[i].end());
      F.brp[i + 1] = F.brp[i] + int(r.size());
    }
    F.bci.reserve(F.brp[nblk]);
    for (int i = 0; i < nblk; ++i) F.bci.insert(F.bci.end(), rows[i].begin(), rows[i].end());
  }
  const int nnzb = F.brp[nblk];
  F.bdiag.resize(nblk);
  for (int i = 0; i < nblk; ++i) {
    F.bdiag[i] = find_blk(F, i, i);
    if (F.bdiag[i] < 0) return "missing diagonal block";
  }
  F.voff.assign(nnzb + 1, 0);
  for (int i = 0; i < nblk; ++i)
    for (int q = F.brp[i]; q < F.brp[i + 1]; ++q)
      F.voff[q + 1] = F.voff[q] + (long long)bsz(i) * bsz(F.bci[q]);
  F.nval = F.voff[nnzb];
  F.doff.assign(nblk + 1, 0);
  for (int i = 0; i < nblk; ++i) F.doff[i + 1] = F.doff[i] + (long long)bsz(i) * bsz(i);
  F.ndinv = F.doff[nblk];
  // ---- update maps, work count, levels
  F.upd_ptr.assign(nnzb + 1, 0);
  std::vector<int> lvl(nblk, 0);
  for (int i = 0; i < nblk; ++i) {
    const int bi = bsz(i);
    F.flops += (long long)bi * bi * bi;
    for (int q = F.brp[i]; q < F.bdiag[i]; ++q) {
      const int k = F.bci[q], bk = bsz(k);
      lvl[i] = std::max(lvl[i], lvl[k] + 1);
      F.nnz_l += (long long)bi * bk;
      F.flops += (long long)bi * bk * bk;
      for (int t = F.bdiag[k] + 1; t < F.brp[k + 1]; ++t) {
        const int J = F.bci[t];
        const int d = find_blk(F, i, J);
        if (d < 0) return "block pattern is not closed under fill";
        F.upd_src.push_back(t);
        F.upd_dst.push_back(d);
        F.flops += (long long)bi * bk * bsz(J);
      }
      F.upd_ptr[q + 1] = (long long)F.upd_src.size();
    }
    for (int q = F.bdiag[i]; q < F.brp[i + 1]; ++q) F.upd_ptr[q + 1] = (long long)F.upd_src.size();
  }
  for (int q = 0; q < nnzb; ++q)
    if (F.upd_ptr[q + 1] < F.upd_ptr[q]) F.upd_ptr[q + 1] = F.upd_ptr[q];
  F.levels = 0;
  for (int i = 0; i < nblk; ++i) F.levels = std::max(F.levels, lvl[i] + 1);
  F.lvl_ptr.assign(F.levels + 1, 0);
  for (int i = 0; i < nblk; ++i) F.lvl_ptr[lvl[i] + 1]++;
  for (int l = 0; l < F.levels; ++l) F.lvl_ptr[l + 1] += F.lvl_ptr[l];
  F.rows.resize(nblk);
  {
    std::vector<int> fill(F.lvl_ptr.begin(), F.lvl_ptr.end() - 1);
    for (int i = 0; i < nblk; ++i) F.rows[fill[lvl[i]]++] = i;
  }
  // ---- assembly maps
  auto slot = [&](int u, int v) -> long long {
    const int I = blk[u], J = blk[v];
    const int q = find_blk(F, I, J);
    if (q < 0) return -1;
    return F.voff[q] + (long long)(F.pos[u] - F.bptr[I]) * bsz(J) + (F.pos[v] - F.bptr[J]);
  };
  {
    // K positions (c-order) that carry W: line-end Hessian blocks, generator
    // cost curvature, slack cost curvature
    std::vector<char> isW(P.K.nnz(), 0);
    for (long long p = 0; p < P.K.nnz(); ++p)
      if (P.Wgat.ptr[p + 1] > P.Wgat.ptr[p] || P.Wgat.cst[p] != 0.0) isW[p] = 1;
    for (int p : P.Wslack_pos) isW[p] = 1;
    for (int wv = 0; wv < nw; ++wv)
      for (int p = P.Knat_rp[wv]; p < P.Knat_rp[wv + 1]; ++p) {
        const int cpos = P.Knat_map[p];
        if (!isW[cpos]) continue;
        const long long s = slot(wv, P.Knat_ci[p]);
        if (s < 0) return "W entry outside the block pattern";
        F.w_slot.push_back(s);
        F.w_src.push_back(cpos);
      }
  }
  for (int r = 0; r < nx; ++r)
    for (int q = P.G.rp[r]; q < P.G.rp[r + 1]; ++q) {
      const int wv = P.G.ci[q];
      const long long s1 = slot(nw + r, wv), s2 = slot(wv, nw + r);
      if (s1 < 0 || s2 < 0) return "G entry outside the block pattern";
      F.g_slot.push_back(s1);
      F.g_src.push_back(q);
      F.g_slot.push_back(s2);
      F.g_src.push_back(q);
    }
  for (int r = 0; r < m; ++r)
    for (int q = P.A.rp[r]; q < P.A.rp[r + 1]; ++q) {
      const int wv = P.A.ci[q];
      const long long s1 = slot(nw + nx + r, wv), s2 = slot(wv, nw + nx + r);
      if (s1 < 0 || s2 < 0) return "A entry outside the block pattern";
      F.a_slot.push_back(s1);
      F.a_src.push_back(q);
      F.a_slot.push_back(s2);
      F.a_src.push_back(q);
    }
  F.diag_slot.resize(n);
  for (int u = 0; u < n; ++u) F.diag_slot[u] = slot(u, u);
  return "";
}

}  // namespace condipm
