// Host-only checks of the full-space symbolic analysis (build_fs_plan): the
// positions form a permutation, the block pattern is symmetric, closed under
// fill and level-ordered, every assembly slot lies inside the value array and
// is written by exactly one source, and the update maps stay inside the rows
// they name.  Reads a network in the binary layout tests/test_plan_host.py
// writes; prints "ok n nblk bmax levels nnzb nval nnz_l flops" or the first
// violation.
#include <cstdio>
#include <string>
#include <vector>

#include "fsplan.h"
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
  FsPlan F;
  e = build_fs_plan(P, F);
  if (!e.empty()) return fail("build_fs_plan: " + e);
  const int n = F.n, nblk = F.nblk;
  if (n != P.nw + P.nx + P.m) return fail("n");
  std::vector<int> seen(n, 0);
  for (int u = 0; u < n; ++u) {
    if (F.pos[u] < 0 || F.pos[u] >= n) return fail("position out of range");
    ++seen[F.pos[u]];
  }
  for (int p = 0; p < n; ++p)
    if (seen[p] != 1) return fail("positions are not a permutation");
  auto bsz = [&](int I) { return F.bptr[I + 1] - F.bptr[I]; };
  auto find = [&](int I, int J) {
    for (int q = F.brp[I]; q < F.brp[I + 1]; ++q)
      if (F.bci[q] == J) return q;
    return -1;
  };
  for (int I = 0; I < nblk; ++I) {
    if (bsz(I) < 1 || bsz(I) > FS_BMAX) return fail("block size");
    for (int q = F.brp[I]; q < F.brp[I + 1]; ++q) {
      if (q > F.brp[I] && F.bci[q] <= F.bci[q - 1]) return fail("row not sorted");
      if ((q < F.bdiag[I]) != (F.bci[q] < I)) return fail("L / U split");
      if (find(F.bci[q], I) < 0) return fail("pattern not symmetric");
      if (F.voff[q + 1] - F.voff[q] != (long long)bsz(I) * bsz(F.bci[q])) return fail("value offsets");
      if (q >= F.bdiag[I] && F.upd_ptr[q + 1] != F.upd_ptr[q]) return fail("update map on a U block");
      for (long long t = F.upd_ptr[q]; t < F.upd_ptr[q + 1]; ++t) {
        const int K = F.bci[q], s = F.upd_src[t], d = F.upd_dst[t];
        if (s <= F.bdiag[K] || s >= F.brp[K + 1]) return fail("update source outside row K's U part");
        if (d < F.brp[I] || d >= F.brp[I + 1] || F.bci[d] != F.bci[s]) return fail("update target");
      }
    }
  }
  // level order: every L-part column comes earlier in the schedule
  std::vector<int> at(nblk, -1);
  for (int t = 0; t < nblk; ++t) {
    if (F.rows[t] < 0 || F.rows[t] >= nblk || at[F.rows[t]] >= 0) return fail("schedule is not a permutation");
    at[F.rows[t]] = t;
  }
  for (int I = 0; I < nblk; ++I)
    for (int q = F.brp[I]; q < F.bdiag[I]; ++q)
      if (at[F.bci[q]] >= at[I]) return fail("schedule not topological");
  // assembly slots: inside the values, one source each
  std::vector<unsigned char> used(F.nval, 0);
  auto mark = [&](const std::vector<long long>& sl) {
    for (long long s : sl) {
      if (s < 0 || s >= F.nval) return false;
      if (used[s]++) return false;
    }
    return true;
  };
  if (!mark(F.w_slot)) return fail("W slot");
  if (!mark(F.g_slot)) return fail("G slot");
  if (!mark(F.a_slot)) return fail("A slot");
  std::vector<unsigned char> dused(F.nval, 0);
  for (int u = 0; u < n; ++u) {
    const long long s = F.diag_slot[u];
    if (s < 0 || s >= F.nval || dused[s]++) return fail("diagonal slot");
    if (u >= P.nw && used[s]) return fail("a multiplier's diagonal has a source");
  }
  std::printf("ok %d %d %d %d %d %lld %lld %lld\n", n, nblk, F.bmax, F.levels, F.brp[nblk], F.nval, F.nnz_l,
              F.flops);
  return 0;
}
