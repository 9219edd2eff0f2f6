// Host-side symbolic analysis (see plan.h).
#include "plan.h"

#include <algorithm>
#include <array>
#include <iterator>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <queue>
#include <set>
#include <utility>

namespace condipm {
namespace {

const double INF = 1e300;

// position of column c inside CSR row i (binary search), -1 if absent
int find_pos(const CSR& M, int i, int c) {
  auto b = M.ci.begin() + M.rp[i], e = M.ci.begin() + M.rp[i + 1];
  auto it = std::lower_bound(b, e, c);
  if (it == e || *it != c) return -1;
  return int(it - M.ci.begin());
}

// CSR from per-row sorted unique column lists
CSR csr_from_rows(int ncols, const std::vector<std::vector<int>>& rows) {
  CSR M;
  M.nrows = int(rows.size());
  M.ncols = ncols;
  M.rp.assign(M.nrows + 1, 0);
  for (int i = 0; i < M.nrows; ++i) M.rp[i + 1] = M.rp[i] + int(rows[i].size());
  M.ci.reserve(M.rp.back());
  for (auto& r : rows) M.ci.insert(M.ci.end(), r.begin(), r.end());
  return M;
}

void sort_unique(std::vector<int>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

// Gather plan from (destination, source) pairs, sorted for a fixed summation order.
Gather gather_from_pairs(int ndst, std::vector<std::pair<int, int>>& pr) {
  std::sort(pr.begin(), pr.end());
  Gather g;
  g.ptr.assign(ndst + 1, 0);
  g.cst.assign(ndst, 0.0);
  for (auto& p : pr) g.ptr[p.first + 1]++;
  for (int i = 0; i < ndst; ++i) g.ptr[i + 1] += g.ptr[i];
  g.idx.resize(pr.size());
  for (size_t q = 0; q < pr.size(); ++q) g.idx[q] = pr[q].second;
  return g;
}

// index of the (a, b) entry, a <= b, of a symmetric 4x4 block stored as 10 values
inline int idx10(int a, int b) {
  if (a > b) std::swap(a, b);
  static const int off[4] = {0, 4, 7, 9};
  return off[a] + (b - a);
}

// Minimum-degree ordering of a weighted graph (weights = unknowns per node),
// eliminating on an explicit elimination graph; ties broken by node index.
std::vector<int> min_degree(int n, std::vector<std::vector<int>> adj, const std::vector<int>& wt) {
  std::vector<long long> deg(n, 0);
  std::vector<char> gone(n, 0);
  for (int v = 0; v < n; ++v)
    for (int a : adj[v]) deg[v] += wt[a];
  using E = std::pair<long long, int>;
  std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
  for (int v = 0; v < n; ++v) pq.push({deg[v], v});
  std::vector<int> order;
  order.reserve(n);
  std::vector<int> tmp;
  while (!pq.empty()) {
    auto [d, v] = pq.top();
    pq.pop();
    if (gone[v] || d != deg[v]) continue;
    gone[v] = 1;
    order.push_back(v);
    std::vector<int> nb;
    for (int a : adj[v])
      if (!gone[a]) nb.push_back(a);
    for (int a : nb) {
      tmp.clear();
      std::set_union(adj[a].begin(), adj[a].end(), nb.begin(), nb.end(), std::back_inserter(tmp));
      std::vector<int> nn;
      nn.reserve(tmp.size());
      for (int c : tmp)
        if (c != a && c != v && !gone[c]) nn.push_back(c);
      adj[a].swap(nn);
      long long dd = 0;
      for (int c : adj[a]) dd += wt[c];
      deg[a] = dd;
      pq.push({dd, a});
    }
    adj[v].clear();
  }
  return order;
}

Levels make_levels(const CSR& M, bool lower) {
  int n = M.nrows;
  std::vector<int> lev(n, 0);
  int nlev = 0;
  if (lower) {
    for (int i = 0; i < n; ++i) {
      int l = 0;
      for (int q = M.rp[i]; q < M.rp[i + 1]; ++q) l = std::max(l, lev[M.ci[q]] + 1);
      lev[i] = l;
      nlev = std::max(nlev, l + 1);
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      int l = 0;
      for (int q = M.rp[i]; q < M.rp[i + 1]; ++q) l = std::max(l, lev[M.ci[q]] + 1);
      lev[i] = l;
      nlev = std::max(nlev, l + 1);
    }
  }
  Levels L;
  L.nlev = n ? nlev : 0;
  L.ptr.assign(L.nlev + 1, 0);
  for (int i = 0; i < n; ++i) L.ptr[lev[i] + 1]++;
  for (int l = 0; l < L.nlev; ++l) L.ptr[l + 1] += L.ptr[l];
  L.rows.resize(n);
  std::vector<int> fill(L.ptr.begin(), L.ptr.end() - 1);
  for (int i = 0; i < n; ++i) L.rows[fill[lev[i]]++] = i;
  return L;
}

// Supernodal schedule for the strict-lower (upper = false) or strict-upper
// pattern M, supernodes given by start offsets.
std::string make_sn_sched(const CSR& M, const std::vector<int>& start, bool upper, SnSched& S) {
  const int n = M.nrows;
  const int ns = int(start.size()) - 1;
  std::vector<int> sn_of(n);
  for (int s = 0; s < ns; ++s)
    for (int i = start[s]; i < start[s + 1]; ++i) sn_of[i] = s;
  S.ext_beg.resize(n); S.ext_end.resize(n); S.int_beg.resize(n);
  std::vector<int> lev(ns, 0);
  std::vector<double> ext_len(ns, 0.0);
  int nlev = 0;
  auto visit = [&](int s) {
    const int f = start[s], w = start[s + 1] - start[s];
    int l = 0;
    for (int r = f; r < f + w; ++r) {
      const int nint = upper ? (f + w - 1 - r) : (r - f);
      const int len = M.rp[r + 1] - M.rp[r];
      if (len < nint) return std::string("supernode diagonal block is not dense");
      if (upper) {
        S.int_beg[r] = M.rp[r];
        S.ext_beg[r] = M.rp[r] + nint;
        S.ext_end[r] = M.rp[r + 1];
        for (int t = 0; t < nint; ++t)
          if (M.ci[M.rp[r] + t] != r + 1 + t) return std::string("supernode diagonal block is not dense");
      } else {
        S.int_beg[r] = M.rp[r + 1] - nint;
        S.ext_beg[r] = M.rp[r];
        S.ext_end[r] = M.rp[r + 1] - nint;
        for (int t = 0; t < nint; ++t)
          if (M.ci[M.rp[r + 1] - nint + t] != f + t) return std::string("supernode diagonal block is not dense");
      }
      for (int q = S.ext_beg[r]; q < S.ext_end[r]; ++q) l = std::max(l, lev[sn_of[M.ci[q]]] + 1);
      ext_len[s] += S.ext_end[r] - S.ext_beg[r];
    }
    lev[s] = l;
    nlev = std::max(nlev, l + 1);
    return std::string();
  };
  if (upper) {
    for (int s = ns - 1; s >= 0; --s) { std::string e = visit(s); if (!e.empty()) return e; }
  } else {
    for (int s = 0; s < ns; ++s) { std::string e = visit(s); if (!e.empty()) return e; }
  }
  S.nlev = ns ? nlev : 0;
  S.lvl_ptr.assign(S.nlev + 1, 0);
  S.lvl_bptr.assign(S.nlev + 1, 0);
  S.lvl_gs.assign(S.nlev, 1);
  S.lvl_wmax.assign(S.nlev, 1);
  S.lvl_ga.assign(S.nlev, 0);
  S.lvl_rptr.assign(S.nlev + 1, 0);
  std::vector<std::vector<int>> small(S.nlev), big(S.nlev);
  for (int s = 0; s < ns; ++s) (start[s + 1] - start[s] > 32 ? big : small)[lev[s]].push_back(s);
  for (int l = 0; l < S.nlev; ++l) {
    int wmax = 1;
    double ext = 0.0;
    long long rows = 0;
    for (int s : small[l]) {
      wmax = std::max(wmax, start[s + 1] - start[s]);
      ext += ext_len[s];
      rows += start[s + 1] - start[s];
    }
    int want = std::max(wmax, rows ? int(std::ceil(ext / rows / 4.0)) : 1);
    int gs = 1;
    while (gs < want && gs < 32) gs <<= 1;
    S.lvl_gs[l] = gs;
    S.lvl_wmax[l] = wmax;
    // rows of the level and lanes per row for their external entries
    long long next = 0, nrows = 0;
    for (auto* grp : {&small[l], &big[l]})
      for (int s2 : *grp)
        for (int r = start[s2]; r < start[s2 + 1]; ++r) {
          S.rows.push_back(r);
          next += S.ext_end[r] - S.ext_beg[r];
          ++nrows;
        }
    S.lvl_rptr[l + 1] = int(S.rows.size());
    if (next > 0) {
      int wantA = int(std::ceil(double(next) / double(nrows) / 8.0));
      int ga = 1;
      while (ga < wantA && ga < 32) ga <<= 1;
      S.lvl_ga[l] = ga;
    }
    for (int s : small[l]) { S.sn_first.push_back(start[s]); S.sn_w.push_back(start[s + 1] - start[s]); }
    for (int s : big[l]) { S.big_first.push_back(start[s]); S.big_w.push_back(start[s + 1] - start[s]); }
    S.lvl_ptr[l + 1] = int(S.sn_first.size());
    S.lvl_bptr[l + 1] = int(S.big_first.size());
  }
  return "";
}

}  // namespace

void build_sn_stream(const CSR& M, const SnSched& S, const std::vector<int>& start, bool upper, bool unit,
                     int budget, SnStream& out) {
  out = SnStream();
  auto al16 = [](long long b) { return (b + 15) & ~15LL; };
  struct Sup { int f, w; };
  // bytes a set of supernodes needs in one chunk
  auto chunk_size = [&](const std::vector<Sup>& sn, long long& nE, long long& nI, int& nA) {
    nE = 0; nI = 0; nA = 0;
    long long nd = 0;
    for (auto& x : sn) {
      for (int r = x.f; r < x.f + x.w; ++r) { nE += S.ext_end[r] - S.ext_beg[r]; ++nA; }
      nI += (long long)x.w * (x.w - 1) / 2;
      nd += x.w;
    }
    const long long nB = sn.size();
    long long b = 80;
    b = al16(b + 4 * (nA + 1)); b = al16(b + 4 * nA); b = al16(b + 4 * nE); b = al16(b + 8 * nE);
    b = al16(b + 4 * nB); b = al16(b + 4 * nB); b = al16(b + 4 * (nB + 1)); b = al16(b + 4 * (nB + 1));
    b = al16(b + 8 * nI); b = al16(b + 8 * nd);
    return b;
  };
  auto emit = [&](const std::vector<Sup>& sn, bool with_b, int ga, int gs, int wmax) {
    long long nE, nI;
    int nA;
    chunk_size(sn, nE, nI, nA);
    if (!with_b) nI = 0;
    const int nB = with_b ? int(sn.size()) : 0;
    long long nd = 0;
    if (with_b) for (auto& x : sn) nd += x.w;
    long long o = 80;
    const long long oAptr = o; o = al16(o + 4LL * (nA + 1));
    const long long oArow = o; o = al16(o + 4LL * nA);
    const long long oEci = o; o = al16(o + 4 * nE);
    const long long oEval = o; o = al16(o + 8 * nE);
    const long long oBf = o; o = al16(o + 4LL * nB);
    const long long oBw = o; o = al16(o + 4LL * nB);
    const long long oBiptr = o; o = al16(o + 4LL * (nB + 1));
    const long long oBdptr = o; o = al16(o + 4LL * (nB + 1));
    const long long oIval = o; o = al16(o + 8 * nI);
    const long long oBd = o; o = al16(o + 8 * nd);
    const long long base = out.bytes.size();
    out.bytes.resize(base + o, 0);
    out.chunk_off.push_back(base);
    out.chunk_bytes.push_back(int(o));
    out.chunk_big_f.push_back(-1);
    out.chunk_big_w.push_back(0);
    out.max_chunk = std::max(out.max_chunk, int(o));
    unsigned char* B = out.bytes.data() + base;
    int hdr[20] = {nA, nB, int(nE), int(nI), ga, gs, wmax, 0, int(oAptr), int(oArow), int(oEci), int(oEval),
                   int(oBf), int(oBw), int(oBiptr), int(oBdptr), int(oIval), int(oBd), 0, 0};
    std::memcpy(B, hdr, sizeof(hdr));
    int* Aptr = reinterpret_cast<int*>(B + oAptr);
    int* Arow = reinterpret_cast<int*>(B + oArow);
    int* Eci = reinterpret_cast<int*>(B + oEci);
    int a = 0, e = 0;
    Aptr[0] = 0;
    std::vector<int> order;
    for (auto& x : sn)
      for (int r = x.f; r < x.f + x.w; ++r) order.push_back(r);
    std::stable_sort(order.begin(), order.end(), [&](int p1, int p2) {
      return S.ext_end[p1] - S.ext_beg[p1] > S.ext_end[p2] - S.ext_beg[p2];
    });
    for (int r : order) {
      Arow[a] = r;
      for (int q = S.ext_beg[r]; q < S.ext_end[r]; ++q, ++e) {
        Eci[e] = M.ci[q];
        out.slot.push_back((base + oEval) / 8 + e);
        out.src.push_back(q);
      }
      Aptr[++a] = e;
    }
    if (!with_b) return;
    int* Bf = reinterpret_cast<int*>(B + oBf);
    int* Bw = reinterpret_cast<int*>(B + oBw);
    int* Biptr = reinterpret_cast<int*>(B + oBiptr);
    int* Bdptr = reinterpret_cast<int*>(B + oBdptr);
    long long ip = 0, dp = 0;
    for (int k = 0; k < nB; ++k) {
      const int f = sn[k].f, w = sn[k].w;
      Bf[k] = f; Bw[k] = w; Biptr[k] = int(ip); Bdptr[k] = int(dp);
      for (int si = 0; si < w; ++si) {
        const int r = f + si;
        const int cnt = upper ? (w - 1 - si) : si;
        const long long off = upper ? ((long long)si * (w - 1) - (long long)si * (si - 1) / 2) : (long long)si * (si - 1) / 2;
        for (int t = 0; t < cnt; ++t) {
          out.slot.push_back((base + oIval) / 8 + ip + off + t);
          out.src.push_back(S.int_beg[r] + t);
        }
        out.slot.push_back((base + oBd) / 8 + dp + si);
        out.src.push_back(unit ? -1 : -2 - r);
      }
      ip += (long long)w * (w - 1) / 2;
      dp += w;
    }
    Biptr[nB] = int(ip);
    Bdptr[nB] = int(dp);
  };
  for (int l = 0; l < S.nlev; ++l) {
    const int ga = std::max(1, S.lvl_ga[l]), gs = S.lvl_gs[l], wmax = S.lvl_wmax[l];
    std::vector<Sup> cur;
    for (int k = S.lvl_ptr[l]; k < S.lvl_ptr[l + 1]; ++k) {
      Sup x{S.sn_first[k], S.sn_w[k]};
      std::vector<Sup> trial = cur;
      trial.push_back(x);
      long long nE, nI;
      int nA;
      if (chunk_size(trial, nE, nI, nA) <= budget) { cur.swap(trial); continue; }
      if (!cur.empty()) { emit(cur, true, ga, gs, wmax); cur.clear(); }
      std::vector<Sup> one{x};
      if (chunk_size(one, nE, nI, nA) <= budget) { cur = one; continue; }
      // a supernode whose rows alone overflow a chunk: its external entries go in
      // row chunks first, its diagonal block in a chunk of its own
      std::vector<Sup> rows;
      for (int r = x.f; r < x.f + x.w; ++r) {
        std::vector<Sup> t2 = rows;
        t2.push_back({r, 1});
        if (!rows.empty() && chunk_size(t2, nE, nI, nA) > budget) { emit(rows, false, 32, 1, 1); rows.clear(); t2 = {{r, 1}}; }
        rows.swap(t2);
      }
      if (!rows.empty()) emit(rows, false, 32, 1, 1);
      // its diagonal block in a chunk without rows (external entries already applied)
      {
        // build the chunk by hand with nA = nE = 0
        const long long nI2 = (long long)x.w * (x.w - 1) / 2;
        long long o = 80;
        const long long oAptr = o; o = al16(o + 4);
        const long long oArow = o;
        const long long oEci = o;
        const long long oEval = o;
        const long long oBf = o; o = al16(o + 4);
        const long long oBw = o; o = al16(o + 4);
        const long long oBiptr = o; o = al16(o + 8);
        const long long oBdptr = o; o = al16(o + 8);
        const long long oIval = o; o = al16(o + 8 * nI2);
        const long long oBd = o; o = al16(o + 8LL * x.w);
        const long long base = out.bytes.size();
        out.bytes.resize(base + o, 0);
        out.chunk_off.push_back(base);
        out.chunk_bytes.push_back(int(o));
        out.chunk_big_f.push_back(-1);
        out.chunk_big_w.push_back(0);
        out.max_chunk = std::max(out.max_chunk, int(o));
        unsigned char* B = out.bytes.data() + base;
        int hdr[20] = {0, 1, 0, int(nI2), 1, gs, wmax, 0, int(oAptr), int(oArow), int(oEci), int(oEval),
                       int(oBf), int(oBw), int(oBiptr), int(oBdptr), int(oIval), int(oBd), 0, 0};
        std::memcpy(B, hdr, sizeof(hdr));
        reinterpret_cast<int*>(B + oAptr)[0] = 0;
        reinterpret_cast<int*>(B + oBf)[0] = x.f;
        reinterpret_cast<int*>(B + oBw)[0] = x.w;
        reinterpret_cast<int*>(B + oBiptr)[0] = 0;
        reinterpret_cast<int*>(B + oBiptr)[1] = int(nI2);
        reinterpret_cast<int*>(B + oBdptr)[0] = 0;
        reinterpret_cast<int*>(B + oBdptr)[1] = x.w;
        for (int si = 0; si < x.w; ++si) {
          const int r = x.f + si;
          const int cnt = upper ? (x.w - 1 - si) : si;
          const long long off = upper ? ((long long)si * (x.w - 1) - (long long)si * (si - 1) / 2)
                                      : (long long)si * (si - 1) / 2;
          for (int t = 0; t < cnt; ++t) {
            out.slot.push_back((base + oIval) / 8 + off + t);
            out.src.push_back(S.int_beg[r] + t);
          }
          out.slot.push_back((base + oBd) / 8 + si);
          out.src.push_back(unit ? -1 : -2 - r);
        }
      }
    }
    if (!cur.empty()) emit(cur, true, ga, gs, wmax);
    // big supernodes: external entries in row chunks, then a big marker chunk
    for (int k = S.lvl_bptr[l]; k < S.lvl_bptr[l + 1]; ++k) {
      const int f = S.big_first[k], w = S.big_w[k];
      std::vector<Sup> rows;
      long long nE, nI;
      int nA;
      for (int r = f; r < f + w; ++r) {
        std::vector<Sup> t2 = rows;
        t2.push_back({r, 1});
        if (!rows.empty() && chunk_size(t2, nE, nI, nA) > budget) { emit(rows, false, 32, 1, 1); rows.clear(); t2 = {{r, 1}}; }
        rows.swap(t2);
      }
      if (!rows.empty()) emit(rows, false, 32, 1, 1);
      out.chunk_off.push_back(out.bytes.size());
      out.chunk_bytes.push_back(0);
      out.chunk_big_f.push_back(f);
      out.chunk_big_w.push_back(w);
    }
  }
}

// column-parallel schedule: supernodes cut to <= 32 rows, long rows in segments
std::string build_col_sched(const CSR& M, const std::vector<int>& sn_start, bool upper, ColSched& C) {
  std::vector<int> start{0};
  for (size_t s = 0; s + 1 < sn_start.size(); ++s)
    for (int f = sn_start[s] + 32; f < sn_start[s + 1]; f += 32) start.push_back(f);
  {
    std::vector<int> all(sn_start.begin() + 1, sn_start.end());
    all.insert(all.end(), start.begin() + 1, start.end());
    std::sort(all.begin(), all.end());
    start.assign(1, 0);
    for (int v : all) if (v != start.back()) start.push_back(v);
  }
  SnSched S;
  std::string e = make_sn_sched(M, start, upper, S);
  if (!e.empty()) return e;
  if (!S.big_first.empty()) return "column schedule has a supernode wider than 32";
  const int SEG = 32;
  C = ColSched();
  C.nlev = S.nlev;
  C.lvl_ptr = S.lvl_ptr;
  C.sn_first = S.sn_first;
  C.sn_w = S.sn_w;
  C.ext_beg = S.ext_beg;
  C.ext_end = S.ext_end;
  C.int_beg = S.int_beg;
  const int n = M.nrows;
  C.row_seg.assign(n, -1);
  C.row_nseg.assign(n, 0);
  C.lvl_seg_ptr.assign(C.nlev + 1, 0);
  for (int l = 0; l < C.nlev; ++l) {
    int slot = 0;
    for (int k = C.lvl_ptr[l]; k < C.lvl_ptr[l + 1]; ++k)
      for (int r = C.sn_first[k]; r < C.sn_first[k] + C.sn_w[k]; ++r) {
        const int len = C.ext_end[r] - C.ext_beg[r];
        if (len == 0) continue;
        const int ns = (len + SEG - 1) / SEG;
        C.row_seg[r] = ns > 1 ? slot : -1;
        C.row_nseg[r] = ns > 1 ? ns : -1;      // -1: one segment, applied to X directly
        for (int q = C.ext_beg[r]; q < C.ext_end[r]; q += SEG) {
          C.seg_q0.push_back(q);
          C.seg_q1.push_back(std::min(q + SEG, C.ext_end[r]));
          C.seg_row.push_back(ns > 1 ? -1 - slot : r);   // >= 0: row to update; < 0: scratch slot
          if (ns > 1) ++slot;
        }
      }
    C.lvl_seg_ptr[l + 1] = int(C.seg_q0.size());
    C.maxseg = std::max(C.maxseg, slot);
  }
  return "";
}

std::string build_plan(Plan& P, int nb, int nl, int ng, int slack, const double* Pd,
                       const double* Qd, const double* Vmin, const double* Vmax,
                       const int* lf, const int* lt, const double* r, const double* x,
                       const double* b, const double* rate, const int* gbus,
                       const double* Pmin, const double* Pmax, const double* Qmin,
                       const double* Qmax, const double* c2, const double* c1) {
  // ---------------------------------------------------------------- checks
  if (nb < 2 || nl < 1 || ng < 1) return "network too small";
  if (!Pd || !Qd || !Vmin || !Vmax || !lf || !lt || !r || !x || !b || !rate || !gbus || !Pmin ||
      !Pmax || !Qmin || !Qmax || !c2 || !c1)
    return "null network array";
  std::vector<int> gen_of_bus(nb, -1);
  for (int k = 0; k < ng; ++k) {
    if (gbus[k] < 0 || gbus[k] >= nb) return "generator bus out of range";
    if (gen_of_bus[gbus[k]] >= 0) return "two generators on one bus";
    gen_of_bus[gbus[k]] = k;
  }
  if (slack != gbus[0]) return "slack must be the bus of generator 0";
  for (int l = 0; l < nl; ++l) {
    if (lf[l] < 0 || lf[l] >= nb || lt[l] < 0 || lt[l] >= nb || lf[l] == lt[l])
      return "bad line endpoints";
    if (!(r[l] * r[l] + x[l] * x[l] > 0)) return "zero line impedance";
  }
  // ---------------------------------------------------------------- copy
  P.nb = nb; P.nl = nl; P.ng = ng; P.slack = slack;
  auto cp = [](const double* a, int n) { return std::vector<double>(a, a + n); };
  P.Pd = cp(Pd, nb); P.Qd = cp(Qd, nb); P.Vmin = cp(Vmin, nb); P.Vmax = cp(Vmax, nb);
  P.r = cp(r, nl); P.x = cp(x, nl); P.b = cp(b, nl); P.rate = cp(rate, nl);
  P.Pmin = cp(Pmin, ng); P.Pmax = cp(Pmax, ng); P.Qmin = cp(Qmin, ng); P.Qmax = cp(Qmax, ng);
  P.c2 = cp(c2, ng); P.c1 = cp(c1, ng);
  P.lf.assign(lf, lf + nl); P.lt.assign(lt, lt + nl); P.gbus.assign(gbus, gbus + ng);
  P.gen_of_bus = gen_of_bus;
  // ---------------------------------------------------------------- layout
  const int nu = 2 * ng - 1;
  const int nload = nb - ng;
  const int nx = (nb - 1) + nload;
  const int nw = nu + nx;
  P.nu = nu; P.nx = nx; P.nw = nw;
  P.th_w.assign(nb, -1); P.vm_w.assign(nb, -1); P.pg_w.assign(ng, -1);
  P.g_row_P.assign(nb, -1); P.g_row_Q.assign(nb, -1);
  {
    int kth = 0, kvm = 0;
    for (int i = 0; i < nb; ++i) {
      if (i != slack) { P.th_w[i] = nu + kth; P.g_row_P[i] = kth; ++kth; }
    }
    for (int i = 0; i < nb; ++i) {
      if (gen_of_bus[i] < 0) { P.vm_w[i] = nu + (nb - 1) + kvm; P.g_row_Q[i] = (nb - 1) + kvm; ++kvm; }
      else P.vm_w[i] = gen_of_bus[i];
    }
    for (int k = 1; k < ng; ++k) P.pg_w[k] = ng + k - 1;
  }
  P.wl.assign(nw, -INF); P.wu.assign(nw, INF);
  for (int i = 0; i < nb; ++i) { P.wl[P.vm_w[i]] = Vmin[i]; P.wu[P.vm_w[i]] = Vmax[i]; }
  for (int k = 1; k < ng; ++k) { P.wl[P.pg_w[k]] = Pmin[k]; P.wu[P.pg_w[k]] = Pmax[k]; }
  std::vector<int> lim;
  for (int l = 0; l < nl; ++l)
    if (rate[l] > 0) lim.push_back(l);
  const int nlim = int(lim.size());
  P.nlim = nlim;
  const int m = 1 + ng + 2 * nlim;
  P.m = m;
  P.hl.assign(m, -INF); P.hu.assign(m, INF);
  P.hl[0] = Pmin[0]; P.hu[0] = Pmax[0];
  for (int k = 0; k < ng; ++k) { P.hl[1 + k] = Qmin[k]; P.hu[1 + k] = Qmax[k]; }
  for (int t = 0; t < nlim; ++t) {
    P.hu[1 + ng + t] = rate[lim[t]] * rate[lim[t]];
    P.hu[1 + ng + nlim + t] = rate[lim[t]] * rate[lim[t]];
  }
  // ---------------------------------------------------------------- ends
  const int ne = 2 * nl;
  P.ne = ne;
  P.end_i.resize(ne); P.end_k.resize(ne); P.end_w.resize(4 * ne); P.end_h.assign(ne, -1);
  P.gs.resize(ne); P.bs.resize(ne); P.gm.resize(ne); P.bm.resize(ne);
  for (int e = 0; e < ne; ++e) {
    int l = e < nl ? e : e - nl;
    int i = e < nl ? lf[l] : lt[l];
    int k = e < nl ? lt[l] : lf[l];
    double d = r[l] * r[l] + x[l] * x[l];
    double gy = r[l] / d, by = -x[l] / d;
    P.end_i[e] = i; P.end_k[e] = k;
    P.gs[e] = gy; P.bs[e] = by + 0.5 * b[l];
    P.gm[e] = -gy; P.bm[e] = -by;
    P.end_w[4 * e + 0] = P.th_w[i];
    P.end_w[4 * e + 1] = P.th_w[k];
    P.end_w[4 * e + 2] = P.vm_w[i];
    P.end_w[4 * e + 3] = P.vm_w[k];
  }
  for (int t = 0; t < nlim; ++t) {
    P.end_h[lim[t]] = 1 + ng + t;
    P.end_h[lim[t] + nl] = 1 + ng + nlim + t;
  }
  P.bus_end_ptr.assign(nb + 1, 0);
  for (int e = 0; e < ne; ++e) P.bus_end_ptr[P.end_i[e] + 1]++;
  for (int i = 0; i < nb; ++i) P.bus_end_ptr[i + 1] += P.bus_end_ptr[i];
  P.bus_end.resize(ne);
  {
    std::vector<int> f(P.bus_end_ptr.begin(), P.bus_end_ptr.end() - 1);
    for (int e = 0; e < ne; ++e) P.bus_end[f[P.end_i[e]]++] = e;
  }
  for (int i = 0; i < nb; ++i)
    if (P.bus_end_ptr[i + 1] == P.bus_end_ptr[i]) return "isolated bus";
  // ---------------------------------------------------------------- G and A
  {
    std::vector<std::vector<int>> rows(nx);
    std::vector<std::pair<std::pair<int, int>, int>> terms;  // ((row, col), src)
    std::vector<std::pair<std::pair<int, int>, double>> csts;
    for (int i = 0; i < nb; ++i) {
      for (int t = P.bus_end_ptr[i]; t < P.bus_end_ptr[i + 1]; ++t) {
        int e = P.bus_end[t];
        for (int l = 0; l < 4; ++l) {
          int wv = P.end_w[4 * e + l];
          if (wv < 0) continue;
          if (P.g_row_P[i] >= 0) { rows[P.g_row_P[i]].push_back(wv); terms.push_back({{P.g_row_P[i], wv}, 4 * e + l}); }
          if (P.g_row_Q[i] >= 0) { rows[P.g_row_Q[i]].push_back(wv); terms.push_back({{P.g_row_Q[i], wv}, 4 * ne + 4 * e + l}); }
        }
      }
      int k = gen_of_bus[i];
      if (k >= 1) { rows[P.g_row_P[i]].push_back(P.pg_w[k]); csts.push_back({{P.g_row_P[i], P.pg_w[k]}, -1.0}); }
    }
    for (auto& rw : rows) sort_unique(rw);
    P.G = csr_from_rows(nw, rows);
    std::vector<std::pair<int, int>> pr;
    for (auto& t : terms) pr.push_back({find_pos(P.G, t.first.first, t.first.second), t.second});
    P.Ggat = gather_from_pairs(int(P.G.nnz()), pr);
    for (auto& c : csts) P.Ggat.cst[find_pos(P.G, c.first.first, c.first.second)] += c.second;
  }
  {
    std::vector<std::vector<int>> rows(m);
    std::vector<std::pair<std::pair<int, int>, int>> terms;
    auto add_bus = [&](int row, int i, int off) {
      for (int t = P.bus_end_ptr[i]; t < P.bus_end_ptr[i + 1]; ++t) {
        int e = P.bus_end[t];
        for (int l = 0; l < 4; ++l) {
          int wv = P.end_w[4 * e + l];
          if (wv < 0) continue;
          rows[row].push_back(wv);
          terms.push_back({{row, wv}, off + 4 * e + l});
        }
      }
    };
    add_bus(0, slack, 0);
    for (int k = 0; k < ng; ++k) add_bus(1 + k, gbus[k], 4 * ne);
    for (int e = 0; e < ne; ++e) {
      if (P.end_h[e] < 0) continue;
      for (int l = 0; l < 4; ++l) {
        int wv = P.end_w[4 * e + l];
        if (wv < 0) continue;
        rows[P.end_h[e]].push_back(wv);
        terms.push_back({{P.end_h[e], wv}, 8 * ne + 4 * e + l});
      }
    }
    for (auto& rw : rows) sort_unique(rw);
    P.A = csr_from_rows(nw, rows);
    std::vector<std::pair<int, int>> pr;
    for (auto& t : terms) pr.push_back({find_pos(P.A, t.first.first, t.first.second), t.second});
    P.Agat = gather_from_pairs(int(P.A.nnz()), pr);
  }
  // ---------------------------------------------------------------- ordering of G_x
  {
    // bus graph over non-slack buses; weight = unknowns per bus
    std::vector<int> bid(nb, -1), bus_of;
    for (int i = 0; i < nb; ++i)
      if (i != slack) { bid[i] = int(bus_of.size()); bus_of.push_back(i); }
    int n = int(bus_of.size());
    std::vector<std::vector<int>> adj(n);
    for (int l = 0; l < nl; ++l) {
      int a = bid[lf[l]], c = bid[lt[l]];
      if (a < 0 || c < 0) continue;
      adj[a].push_back(c);
      adj[c].push_back(a);
    }
    for (auto& a : adj) sort_unique(a);
    std::vector<int> wt(n);
    for (int v = 0; v < n; ++v) wt[v] = gen_of_bus[bus_of[v]] >= 0 ? 1 : 2;
    std::vector<int> ord = min_degree(n, adj, wt);
    P.perm.clear();
    for (int v : ord) {
      int i = bus_of[v];
      P.perm.push_back(P.th_w[i] - nu);
      if (gen_of_bus[i] < 0) P.perm.push_back(P.vm_w[i] - nu);
    }
    if (int(P.perm.size()) != nx) return "ordering size mismatch";
    P.iperm.assign(nx, -1);
    for (int k = 0; k < nx; ++k) P.iperm[P.perm[k]] = k;
  }
  P.w2c.resize(nw); P.c2w.resize(nw);
  for (int v = 0; v < nu; ++v) P.w2c[v] = v;
  for (int j = 0; j < nx; ++j) P.w2c[nu + j] = nu + P.iperm[j];
  for (int v = 0; v < nw; ++v) P.c2w[P.w2c[v]] = v;
  // ---------------------------------------------------------------- symbolic LU
  {
    const int n = nx;
    std::vector<std::vector<int>> adj(n);
    for (int rr = 0; rr < nx; ++rr)
      for (int q = P.G.rp[rr]; q < P.G.rp[rr + 1]; ++q) {
        int c = P.G.ci[q];
        if (c < nu) continue;
        int pi = P.iperm[rr], pj = P.iperm[c - nu];
        if (pi == pj) continue;
        adj[pi].push_back(pj);
        adj[pj].push_back(pi);
      }
    for (auto& a : adj) sort_unique(a);
    std::vector<std::vector<int>> Ls(n), children(n);
    std::vector<int> mark(n, -1);
    for (int j = 0; j < n; ++j) {
      std::vector<int>& s = Ls[j];
      for (int i : adj[j])
        if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
      for (int c : children[j])
        for (int i : Ls[c])
          if (i > j && mark[i] != j) { mark[i] = j; s.push_back(i); }
      std::sort(s.begin(), s.end());
      if (!s.empty()) children[s[0]].push_back(j);
    }
    // combined rows: L part (transposed column structures), diagonal, U part
    std::vector<std::vector<int>> rows(n);
    for (int j = 0; j < n; ++j)
      for (int i : Ls[j]) rows[i].push_back(j);
    for (int i = 0; i < n; ++i) {
      rows[i].push_back(i);
      rows[i].insert(rows[i].end(), Ls[i].begin(), Ls[i].end());
    }
    P.LU = csr_from_rows(n, rows);
    P.LU_diag.resize(n);
    for (int i = 0; i < n; ++i) P.LU_diag[i] = find_pos(P.LU, i, i);
    // update map of every L entry (i, k): positions of (i, j) for j in U(k), j > k
    P.upd_ptr.assign(P.LU.nnz() + 1, 0);
    long long total = 0;
    for (int i = 0; i < n; ++i) {
      for (int q = P.LU.rp[i]; q < P.LU.rp[i + 1]; ++q) {
        int k = P.LU.ci[q];
        long long len = (k < i) ? (P.LU.rp[k + 1] - P.LU_diag[k] - 1) : 0;
        P.upd_ptr[q + 1] = len;
        total += len;
      }
    }
    for (size_t q = 0; q + 1 < P.upd_ptr.size(); ++q) P.upd_ptr[q + 1] += P.upd_ptr[q];
    P.upd_pos.resize(total);
    for (int i = 0; i < n; ++i) {
      for (int q = P.LU.rp[i]; q < P.LU_diag[i]; ++q) {
        int k = P.LU.ci[q];
        long long base = P.upd_ptr[q];
        for (int t = P.LU_diag[k] + 1; t < P.LU.rp[k + 1]; ++t) {
          int pos = find_pos(P.LU, i, P.LU.ci[t]);
          if (pos < 0) return "symbolic LU pattern is not closed under fill";
          P.upd_pos[base + (t - P.LU_diag[k] - 1)] = pos;
        }
      }
    }
    P.lu_flops = total + (P.LU.nnz() - n) / 2;
    // strict lower / upper views
    std::vector<std::vector<int>> lo(n), up(n);
    for (int i = 0; i < n; ++i)
      for (int q = P.LU.rp[i]; q < P.LU.rp[i + 1]; ++q) {
        int c = P.LU.ci[q];
        if (c < i) lo[i].push_back(c);
        else if (c > i) up[i].push_back(c);
      }
    P.Lo = csr_from_rows(n, lo);
    P.Up = csr_from_rows(n, up);
    P.Lo_map.resize(P.Lo.nnz()); P.Ut_map.resize(P.Lo.nnz());
    P.Up_map.resize(P.Up.nnz()); P.Lt_map.resize(P.Up.nnz());
    for (int i = 0; i < n; ++i) {
      for (int q = P.Lo.rp[i]; q < P.Lo.rp[i + 1]; ++q) {
        int j = P.Lo.ci[q];
        P.Lo_map[q] = find_pos(P.LU, i, j);
        P.Ut_map[q] = find_pos(P.LU, j, i);  // U^T(i, j) = U(j, i)
        if (P.Lo_map[q] < 0 || P.Ut_map[q] < 0) return "asymmetric LU pattern";
      }
      for (int q = P.Up.rp[i]; q < P.Up.rp[i + 1]; ++q) {
        int j = P.Up.ci[q];
        P.Up_map[q] = find_pos(P.LU, i, j);
        P.Lt_map[q] = find_pos(P.LU, j, i);  // L^T(i, j) = L(j, i)
        if (P.Up_map[q] < 0 || P.Lt_map[q] < 0) return "asymmetric LU pattern";
      }
    }
    P.fwd = make_levels(P.Lo, true);
    P.bwd = make_levels(P.Up, false);
    // fundamental supernodes: column j joins j-1 when parent(j-1) = j and
    // struct(L(:, j-1)) = {j} + struct(L(:, j)); the diagonal block is then dense
    P.sn_start.assign(1, 0);
    for (int j = 1; j < n; ++j) {
      const int lp = P.Up.rp[j] - P.Up.rp[j - 1];
      const int lj = P.Up.rp[j + 1] - P.Up.rp[j];
      const bool merge = lp > 0 && P.Up.ci[P.Up.rp[j - 1]] == j && lp == lj + 1;
      if (!merge) P.sn_start.push_back(j);
    }
    P.sn_start.push_back(n);
    std::string e1 = make_sn_sched(P.Lo, P.sn_start, false, P.snL);
    if (!e1.empty()) return e1;
    std::string e2 = make_sn_sched(P.Up, P.sn_start, true, P.snU);
    if (!e2.empty()) return e2;
    build_sn_stream(P.Lo, P.snL, P.sn_start, false, false, 32 * 1024, P.stL);
    build_sn_stream(P.Up, P.snU, P.sn_start, true, false, 32 * 1024, P.stU);
    std::string e3 = build_col_sched(P.Lo, P.sn_start, false, P.csL);
    if (!e3.empty()) return e3;
    std::string e4 = build_col_sched(P.Up, P.sn_start, true, P.csU);
    if (!e4.empty()) return e4;
    // G_x entries -> LU positions
    P.Gx_to_LU.assign(P.G.nnz(), -1);
    for (int rr = 0; rr < nx; ++rr)
      for (int q = P.G.rp[rr]; q < P.G.rp[rr + 1]; ++q) {
        int c = P.G.ci[q];
        if (c < nu) continue;
        P.Gx_to_LU[q] = find_pos(P.LU, P.iperm[rr], P.iperm[c - nu]);
        if (P.Gx_to_LU[q] < 0) return "G_x entry outside the LU pattern";
      }
  }
  // ---------------------------------------------------------------- P G_u and (P G_u)^T
  {
    std::vector<std::vector<std::pair<int, int>>> rows(nx), trows(nu);
    for (int rr = 0; rr < nx; ++rr)
      for (int q = P.G.rp[rr]; q < P.G.rp[rr + 1]; ++q) {
        int c = P.G.ci[q];
        if (c >= nu) continue;
        rows[P.iperm[rr]].push_back({c, q});
        trows[c].push_back({P.iperm[rr], q});
      }
    auto build = [](CSR& M, std::vector<int>& map, int ncols,
                    std::vector<std::vector<std::pair<int, int>>>& rw) {
      M.nrows = int(rw.size());
      M.ncols = ncols;
      M.rp.assign(M.nrows + 1, 0);
      for (int i = 0; i < M.nrows; ++i) {
        std::sort(rw[i].begin(), rw[i].end());
        M.rp[i + 1] = M.rp[i] + int(rw[i].size());
        for (auto& p : rw[i]) { M.ci.push_back(p.first); map.push_back(p.second); }
      }
    };
    build(P.PGu, P.PGu_map, nu, rows);
    build(P.GuT, P.GuT_map, nx, trows);
    // all of G with rows in elimination order and columns in c-order, and its
    // transpose: the G and G^T products of the full K_aug residual
    std::vector<std::vector<std::pair<int, int>>> grows(nx), gtrows(nw);
    for (int rr = 0; rr < nx; ++rr)
      for (int q = P.G.rp[rr]; q < P.G.rp[rr + 1]; ++q) {
        const int cc = P.w2c[P.G.ci[q]];
        grows[P.iperm[rr]].push_back({cc, q});
        gtrows[cc].push_back({P.iperm[rr], q});
      }
    build(P.Gc, P.Gc_map, nw, grows);
    build(P.GcT, P.GcT_map, nx, gtrows);
  }
  // ---------------------------------------------------------------- K pattern (c-order)
  {
    std::vector<std::vector<int>> rows(nw);
    for (int c = 0; c < nw; ++c) rows[c].push_back(c);
    for (int e = 0; e < ne; ++e)
      for (int a = 0; a < 4; ++a)
        for (int bb = 0; bb < 4; ++bb) {
          int wa = P.end_w[4 * e + a], wb = P.end_w[4 * e + bb];
          if (wa >= 0 && wb >= 0) rows[P.w2c[wa]].push_back(P.w2c[wb]);
        }
    for (int rr = 0; rr < m; ++rr)
      for (int q = P.A.rp[rr]; q < P.A.rp[rr + 1]; ++q)
        for (int q2 = P.A.rp[rr]; q2 < P.A.rp[rr + 1]; ++q2)
          rows[P.w2c[P.A.ci[q]]].push_back(P.w2c[P.A.ci[q2]]);
    for (auto& rw : rows) sort_unique(rw);
    P.K = csr_from_rows(nw, rows);
    P.K_diag.resize(nw);
    for (int c = 0; c < nw; ++c) P.K_diag[c] = find_pos(P.K, c, c);
    // W gather: Hw[10 e + idx10(a, b)]
    std::vector<std::pair<int, int>> pr;
    for (int e = 0; e < ne; ++e)
      for (int a = 0; a < 4; ++a)
        for (int bb = 0; bb < 4; ++bb) {
          int wa = P.end_w[4 * e + a], wb = P.end_w[4 * e + bb];
          if (wa >= 0 && wb >= 0) pr.push_back({find_pos(P.K, P.w2c[wa], P.w2c[wb]), 10 * e + idx10(a, bb)});
        }
    P.Wgat = gather_from_pairs(int(P.K.nnz()), pr);
    for (int k = 1; k < ng; ++k) {
      int c = P.w2c[P.pg_w[k]];
      P.Wgat.cst[P.K_diag[c]] += 2.0 * c2[k];
    }
    // slack cost curvature 2 c2_0 dP_s dP_s^T on the support of A's row 0
    for (int q = P.A.rp[0]; q < P.A.rp[1]; ++q)
      for (int q2 = P.A.rp[0]; q2 < P.A.rp[1]; ++q2) {
        P.Wslack_pos.push_back(find_pos(P.K, P.w2c[P.A.ci[q]], P.w2c[P.A.ci[q2]]));
        P.Wslack_a.push_back(q);
        P.Wslack_b.push_back(q2);
      }
    // A^T Sigma_s A bilinear terms
    std::vector<std::array<int, 4>> t4;
    for (int rr = 0; rr < m; ++rr)
      for (int q = P.A.rp[rr]; q < P.A.rp[rr + 1]; ++q)
        for (int q2 = P.A.rp[rr]; q2 < P.A.rp[rr + 1]; ++q2)
          t4.push_back({find_pos(P.K, P.w2c[P.A.ci[q]], P.w2c[P.A.ci[q2]]), rr, q, q2});
    std::sort(t4.begin(), t4.end());
    P.KAA.ptr.assign(P.K.nnz() + 1, 0);
    for (auto& t : t4) P.KAA.ptr[t[0] + 1]++;
    for (long long p = 0; p < P.K.nnz(); ++p) P.KAA.ptr[p + 1] += P.KAA.ptr[p];
    for (auto& t : t4) { P.KAA.r.push_back(t[1]); P.KAA.a.push_back(t[2]); P.KAA.b.push_back(t[3]); }
    // natural-order view of K
    P.Knat_rp.assign(nw + 1, 0);
    for (int wv = 0; wv < nw; ++wv) {
      int c = P.w2c[wv];
      std::vector<std::pair<int, int>> ent;
      for (int q = P.K.rp[c]; q < P.K.rp[c + 1]; ++q) ent.push_back({P.c2w[P.K.ci[q]], q});
      std::sort(ent.begin(), ent.end());
      for (auto& pq : ent) { P.Knat_ci.push_back(pq.first); P.Knat_map.push_back(pq.second); }
      P.Knat_rp[wv + 1] = int(P.Knat_ci.size());
    }
  }
  // ---------------------------------------------------------------- G^T, A^T (natural order)
  {
    auto transpose = [&](const CSR& M, CSR& T, std::vector<int>& map) {
      std::vector<std::vector<std::pair<int, int>>> rw(nw);
      for (int rr = 0; rr < M.nrows; ++rr)
        for (int q = M.rp[rr]; q < M.rp[rr + 1]; ++q) rw[M.ci[q]].push_back({rr, q});
      T.nrows = nw;
      T.ncols = M.nrows;
      T.rp.assign(nw + 1, 0);
      T.ci.clear();
      map.clear();
      for (int c = 0; c < nw; ++c) {
        T.rp[c + 1] = T.rp[c] + int(rw[c].size());
        for (auto& p2 : rw[c]) { T.ci.push_back(p2.first); map.push_back(p2.second); }
      }
    };
    transpose(P.G, P.GTn, P.GTn_map);
    transpose(P.A, P.ATn, P.ATn_map);
  }
  // ---------------------------------------------------------------- A in c-order, A^T
  {
    P.A_ci_c.resize(P.A.nnz());
    for (long long q = 0; q < P.A.nnz(); ++q) P.A_ci_c[q] = P.w2c[P.A.ci[q]];
    std::vector<std::vector<std::pair<int, int>>> rw(nw);
    for (int rr = 0; rr < m; ++rr)
      for (int q = P.A.rp[rr]; q < P.A.rp[rr + 1]; ++q) rw[P.w2c[P.A.ci[q]]].push_back({rr, q});
    P.AT.nrows = nw;
    P.AT.ncols = m;
    P.AT.rp.assign(nw + 1, 0);
    for (int c = 0; c < nw; ++c) {
      std::sort(rw[c].begin(), rw[c].end());
      P.AT.rp[c + 1] = P.AT.rp[c] + int(rw[c].size());
      for (auto& p : rw[c]) { P.AT.ci.push_back(p.first); P.AT_map.push_back(p.second); }
    }
  }
  return "";
}


std::string build_cl_sched(const ColSched& C, int CL, ClSched& S) {
  S = ClSched();
  S.CL = CL;
  S.nlev = C.nlev;
  const int ns = int(C.sn_first.size());
  if (CL < 1 || CL > 16) return "bad cluster size";
  std::vector<int> doff(ns + 1, 0), owner(ns, 0);
  for (int q = 0; q < ns; ++q) doff[q + 1] = doff[q] + C.sn_w[q] * C.sn_w[q];
  // owners: per level, largest work first to the least loaded CTA
  for (int l = 0; l < C.nlev; ++l) {
    std::vector<std::pair<long long, int>> work;
    for (int q = C.lvl_ptr[l]; q < C.lvl_ptr[l + 1]; ++q) {
      long long wk = (long long)C.sn_w[q] * C.sn_w[q];
      for (int r = C.sn_first[q]; r < C.sn_first[q] + C.sn_w[q]; ++r) wk += C.ext_end[r] - C.ext_beg[r];
      work.push_back({wk, q});
    }
    std::stable_sort(work.begin(), work.end(), [](const std::pair<long long, int>& a,
                                                  const std::pair<long long, int>& b) { return a.first > b.first; });
    std::vector<long long> load(CL, 0);
    for (const auto& wq : work) {
      int best = 0;
      for (int p = 1; p < CL; ++p)
        if (load[p] < load[best]) best = p;
      owner[wq.second] = best;
      load[best] += wq.first;
    }
  }
  const int L1 = C.nlev + 1;
  S.t_ptr.assign(size_t(CL) * L1, 0);
  auto push4 = [](std::vector<int>& v, int a, int b, int c, int d) {
    v.push_back(a); v.push_back(b); v.push_back(c); v.push_back(d);
  };
  for (int p = 0; p < CL; ++p) {
    for (int l = 0; l < C.nlev; ++l) {
      S.t_ptr[p * L1 + l] = int(S.ta.size() / 4);
      int ycount = 0;
      for (int q = C.lvl_ptr[l]; q < C.lvl_ptr[l + 1]; ++q) {
        if (owner[q] != p) continue;
        const int f = C.sn_first[q], w = C.sn_w[q];
        for (int r = f; r < f + w; ++r) {
          push4(S.ta, r, C.ext_beg[r], C.ext_end[r], ycount + (r - f));
          push4(S.tb, r, ycount, w, doff[q] + (r - f) * w);
        }
        ycount += w;
      }
      S.ymax = std::max(S.ymax, ycount);
    }
    S.t_ptr[p * L1 + C.nlev] = int(S.ta.size() / 4);
  }
  return "";
}
void build_forward_reach(const Plan& P, const ColSched& C, std::vector<int>& ptr, std::vector<int>& q,
                         double work[2]) {
  const int n = P.nx, nblk = P.nu / 32, nlev = C.nlev;
  ptr.assign((size_t)nblk * (nlev + 1), 0);
  q.clear();
  work[0] = work[1] = 0.0;
  // rows in level order, with their supernode
  std::vector<int> rows, rsn;
  for (int l = 0; l < nlev; ++l)
    for (int s = C.lvl_ptr[l]; s < C.lvl_ptr[l + 1]; ++s)
      for (int r = C.sn_first[s]; r < C.sn_first[s] + C.sn_w[s]; ++r) { rows.push_back(r); rsn.push_back(s); }
  auto row_work = [&](int r, int s) {
    return double(C.ext_end[r] - C.ext_beg[r]) + double(r - C.sn_first[s] + 1);
  };
  for (size_t t = 0; t < rows.size(); ++t) work[1] += row_work(rows[t], rsn[t]);
  work[1] *= 32.0 * nblk;
  // the reach of 64 blocks at a time, one bit per block: rows ascend in the
  // elimination order, so one pass over L's rows reaches every row
  std::vector<unsigned long long> in(n);
  for (int b = 0; b < nblk; ++b) {
    const unsigned long long bit = 1ULL << (b & 63);
    if ((b & 63) == 0) {
      const int b0 = b;
      for (int i = 0; i < n; ++i) {
        unsigned long long v = 0;
        for (int e = P.PGu.rp[i]; e < P.PGu.rp[i + 1]; ++e) {
          const int cb = P.PGu.ci[e] / 32 - b0;
          if (cb >= 0 && cb < 64) v |= 1ULL << cb;
        }
        for (int e = P.Lo.rp[i]; e < P.Lo.rp[i + 1]; ++e) v |= in[P.Lo.ci[e]];
        in[i] = v;
      }
    }
    int* bp = &ptr[(size_t)b * (nlev + 1)];
    bp[0] = int(q.size());
    size_t t = 0;
    for (int l = 0; l < nlev; ++l) {
      for (int s = C.lvl_ptr[l]; s < C.lvl_ptr[l + 1]; ++s) {
        const int f = C.sn_first[s], w = C.sn_w[s];
        bool any = false;
        for (int r = f; r < f + w; ++r) any = any || (in[r] & bit) != 0;
        for (int r = f; r < f + w; ++r, ++t)
          if (any) {
            q.push_back(int(t));
            work[0] += 32.0 * row_work(r, s);
          }
      }
      bp[l + 1] = int(q.size());
    }
  }
}

std::vector<int> min_degree_order(int n, const std::vector<std::vector<int>>& adj, const std::vector<int>& wt) {
  return min_degree(n, adj, wt);
}

}  // namespace condipm
