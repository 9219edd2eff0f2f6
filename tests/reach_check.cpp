// Host-only checks of the forward sweep's reach lists (build_forward_reach):
// with random values on the L and P G_u patterns, every row where the computed
// Y = L^{-1} P G_u is nonzero in a 32-column block's columns is on that block's
// list; every listed row is such a row or shares a supernode with one; the
// lists ascend and each level's part lies inside that level's rows; and the
// work counts add up.  Reads a network in the binary layout
// tests/test_plan_host.py writes; prints "ok nblk listed_rows all_rows
// work_fraction" or the first violation.
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "plan.h"

using namespace condipm;

static int fail(const std::string& m) {
  std::printf("FAIL %s\n", m.c_str());
  return 1;
}

int main(int argc, char** argv) {
  if (argc < 2) return fail("usage");
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return fail("open");
  int hd[4];
  if (std::fread(hd, 4, 4, f) != 4) return fail("header");
  const int nb = hd[0], nl = hd[1], ng = hd[2], slack = hd[3];
  auto rd = [&](int n) { std::vector<double> v(n); if (std::fread(v.data(), 8, n, f) != size_t(n)) v.clear(); return v; };
  auto ri = [&](int n) { std::vector<int> v(n); if (std::fread(v.data(), 4, n, f) != size_t(n)) v.clear(); return v; };
  auto Pd = rd(nb), Qd = rd(nb), Vmin = rd(nb), Vmax = rd(nb);
  auto lf = ri(nl), lt = ri(nl);
  auto r = rd(nl), x = rd(nl), b = rd(nl), rate = rd(nl);
  auto gbus = ri(ng);
  auto Pmin = rd(ng), Pmax = rd(ng), Qmin = rd(ng), Qmax = rd(ng), c2 = rd(ng), c1 = rd(ng);
  std::fclose(f);
  Plan P;
  std::string e = build_plan(P, nb, nl, ng, slack, Pd.data(), Qd.data(), Vmin.data(), Vmax.data(), lf.data(),
                             lt.data(), r.data(), x.data(), b.data(), rate.data(), gbus.data(), Pmin.data(),
                             Pmax.data(), Qmin.data(), Qmax.data(), c2.data(), c1.data());
  if (!e.empty()) return fail("build_plan: " + e);
  const ColSched& C = P.csL;
  const int n = P.nx, nu = P.nu, nblk = nu / 32, nlev = C.nlev;
  long long listed = 0, all = 0;
  std::vector<int> ptr, q;
  double work[2];
  build_forward_reach(P, C, ptr, q, work);
  if (ptr.size() != size_t(nblk) * (nlev + 1)) return fail("offset array size");
  // rows in level order, each with its supernode, and each level's range
  std::vector<int> rows, rsn, lvl(nlev + 1, 0);
  for (int l = 0; l < nlev; ++l) {
    for (int s = C.lvl_ptr[l]; s < C.lvl_ptr[l + 1]; ++s)
      for (int rr = C.sn_first[s]; rr < C.sn_first[s] + C.sn_w[s]; ++rr) { rows.push_back(rr); rsn.push_back(s); }
    lvl[l + 1] = int(rows.size());
  }
  if (int(rows.size()) != n) return fail("level order does not cover the rows");
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(0.5, 1.5);
  std::vector<double> Lv(P.Lo.ci.size());
  for (auto& v : Lv) v = U(g) * (g() & 1 ? 1.0 : -1.0) / 4.0;
  std::vector<double> Gv(P.PGu.ci.size());
  for (auto& v : Gv) v = U(g);
  double wsum = 0.0;
  for (int bk = 0; bk < nblk; ++bk) {
    // Y = L^{-1} R for the block's 32 columns, R = random values on P G_u's pattern
    std::vector<double> Y((size_t)n * 32, 0.0);
    for (int i = 0; i < n; ++i) {
      double* y = &Y[(size_t)i * 32];
      for (int t = P.PGu.rp[i]; t < P.PGu.rp[i + 1]; ++t) {
        const int c = P.PGu.ci[t] - 32 * bk;
        if (c >= 0 && c < 32) y[c] += Gv[t];
      }
      for (int t = P.Lo.rp[i]; t < P.Lo.rp[i + 1]; ++t) {
        const double* yj = &Y[(size_t)P.Lo.ci[t] * 32];
        for (int c = 0; c < 32; ++c) y[c] -= Lv[t] * yj[c];
      }
    }
    std::vector<char> nz(n, 0), on(n, 0), sn_nz(C.sn_first.size(), 0);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 32; ++c)
        if (Y[(size_t)i * 32 + c] != 0.0) nz[i] = 1;
    for (int t = 0; t < n; ++t)
      if (nz[rows[t]]) sn_nz[rsn[t]] = 1;
    const int* bp = &ptr[(size_t)bk * (nlev + 1)];
    for (int l = 0; l < nlev; ++l) {
      if (bp[l + 1] < bp[l]) return fail("offsets decrease");
      for (int k = bp[l]; k < bp[l + 1]; ++k) {
        const int t = q[k];
        if (t < lvl[l] || t >= lvl[l + 1]) return fail("listed position outside its level");
        if (k > bp[l] && t <= q[k - 1]) return fail("list does not ascend");
        if (!sn_nz[rsn[t]]) return fail("listed row in a supernode without a nonzero row");
        on[rows[t]] = 1;
        wsum += 32.0 * (double(C.ext_end[rows[t]] - C.ext_beg[rows[t]]) + double(rows[t] - C.sn_first[rsn[t]] + 1));
      }
    }
    if (bk + 1 < nblk && bp[nlev] != ptr[(size_t)(bk + 1) * (nlev + 1)]) return fail("blocks are not contiguous");
    for (int i = 0; i < n; ++i) {
      if (nz[i] && !on[i]) return fail("row with a nonzero solution is not listed, block " + std::to_string(bk));
      listed += on[i];
    }
    for (int t = 0; t < n; ++t)
      if (on[rows[t]] != sn_nz[rsn[t]]) return fail("supernode listed in part");
    all += n;
  }
  if (nblk > 0 && std::fabs(wsum - work[0]) > 1e-9 * work[0]) return fail("listed work count");
  std::printf("ok %d %lld %lld %.6f\n", nblk, listed, all, nblk > 0 ? work[0] / work[1] : 0.0);
  return 0;
}
