// Host-only checks of the symbolic analysis's schedules for the cluster
// one-right-hand-side solve (build_cl_sched): for every factor and cluster size,
// each row of each level is scheduled exactly once for both phases, by the CTA
// that owns its supernode, with Y slots that stay inside the CTA's buffer and
// keep a supernode's rows consecutive.  Reads a network in the binary layout
// tests/test_plan_host.py writes; prints "ok" or the first violation.
#include <cstdio>
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
  const std::string e = build_plan(P, nb, nl, ng, slack, Pd.data(), Qd.data(), Vmin.data(), Vmax.data(), lf.data(),
                                   lt.data(), r.data(), x.data(), b.data(), rate.data(), gbus.data(), Pmin.data(),
                                   Pmax.data(), Qmin.data(), Qmax.data(), c2.data(), c1.data());
  if (!e.empty()) return fail("build_plan: " + e);
  for (int k = 0; k < 2; ++k) {
    const ColSched& C = k ? P.csU : P.csL;
    std::vector<int> lev_of(P.nx, -1), sn_of(P.nx, -1);
    for (int l = 0; l < C.nlev; ++l)
      for (int q = C.lvl_ptr[l]; q < C.lvl_ptr[l + 1]; ++q)
        for (int i = C.sn_first[q]; i < C.sn_first[q] + C.sn_w[q]; ++i) { lev_of[i] = l; sn_of[i] = q; }
    for (int CL : {1, 4, 8, 16}) {
      ClSched S;
      const std::string es = build_cl_sched(C, CL, S);
      if (!es.empty()) return fail("build_cl_sched: " + es);
      const int L1 = S.nlev + 1;
      if (S.nlev != C.nlev || (int)S.t_ptr.size() != CL * L1) return fail("sizes");
      std::vector<int> seen_a(P.nx, 0), seen_b(P.nx, 0), owner(C.sn_first.size(), -1);
      for (int p = 0; p < CL; ++p)
        for (int l = 0; l < S.nlev; ++l) {
          const int t0 = S.t_ptr[p * L1 + l], t1 = S.t_ptr[p * L1 + l + 1];
          if (t1 < t0) return fail("t_ptr not monotone");
          for (int t = t0; t < t1; ++t) {
            const int ra = S.ta[4 * t], rb = S.tb[4 * t];
            if (ra < 0 || ra >= P.nx || rb < 0 || rb >= P.nx) return fail("row out of range");
            if (lev_of[ra] != l || lev_of[rb] != l) return fail("row in the wrong level");
            ++seen_a[ra];
            ++seen_b[rb];
            if (S.ta[4 * t + 1] != C.ext_beg[ra] || S.ta[4 * t + 2] != C.ext_end[ra]) return fail("external range");
            const int q = sn_of[rb], fr = C.sn_first[q], w = C.sn_w[q];
            if (owner[q] < 0) owner[q] = p;
            if (owner[q] != p || (owner[sn_of[ra]] != -1 && owner[sn_of[ra]] != p)) return fail("supernode split over CTAs");
            if (S.tb[4 * t + 2] != w) return fail("width");
            const int y0 = S.tb[4 * t + 1];
            if (y0 < 0 || y0 + w > S.ymax) return fail("Y slots outside the buffer");
            if (S.ta[4 * t + 3] < 0 || S.ta[4 * t + 3] >= S.ymax) return fail("Y slot outside the buffer");
            // the row's own phase-A slot is its supernode's first slot plus its offset
            if (ra == rb && S.ta[4 * t + 3] != y0 + (rb - fr)) return fail("Y slot of the row");
          }
        }
      for (int i = 0; i < P.nx; ++i)
        if (seen_a[i] != 1 || seen_b[i] != 1) return fail("row not scheduled exactly once");
    }
  }
  std::printf("ok\n");
  return 0;
}
