// Host build of the colour-split layout's per-slot functions (the FP32 finest
// level of the mixed viscous solve, hb_visc_split.cuh), checked bit for bit
// against the natural-layout functions the other kernels run, on seeded
// fields: the slot map (every cell of a colour once), each component's
// red-black sweep, the operator with and without a right-hand side, the cell
// restriction and prolongation from and to the split level (all axes even),
// and the FP64 <-> FP32 conversions.  No GPU needed.
//
// argv: n0 n1 n2 hom seed.  Exit 0 when everything agrees, 3 (with a message
// on stderr) at the first difference.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "hb_internal.h"
#include "hb_visc_split.cuh"

using namespace hb;

static unsigned long long g_state = 1;
static double urand() {  // 53-bit uniform in [0, 1) from a 64-bit LCG
  g_state = g_state * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(g_state >> 11) * (1.0 / 9007199254740992.0);
}

static int fail(const char* what) {
  std::fprintf(stderr, "split layout differs: %s\n", what);
  return 3;
}

template <typename T>
static std::vector<T> to_split(const Geom& g, const std::vector<T>& nat, int ncomp) {
  std::vector<T> s(nat.size());
  for (int c = 0; c < ncomp; ++c)
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i)
          s[(size_t)c * g.ncell + sidx(g, i, j, k)] = nat[(size_t)c * g.ncell + cidx<3>(g, i, j, k)];
  return s;
}

template <typename T>
static bool same_split(const Geom& g, const std::vector<T>& nat, const std::vector<T>& spl, int ncomp) {
  const std::vector<T> s = to_split(g, nat, ncomp);
  return std::memcmp(s.data(), spl.data(), s.size() * sizeof(T)) == 0;
}

int main(int argc, char** argv) {
  if (argc != 6) return 1;
  Geom g;
  std::memset(&g, 0, sizeof g);
  for (int a = 0; a < 3; ++a) g.n[a] = std::atoi(argv[1 + a]);
  const int hom = std::atoi(argv[4]);
  g_state = (unsigned long long)std::atoll(argv[5]) * 2654435761ull + 12345ull;
  if (g.n[0] % 2 || g.n[0] < 4 || g.n[1] < 3 || g.n[2] < 3) return 1;
  g.h = 1.0 / g.n[0];
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  g.nnode = (g.n[0] + 1) * (g.n[1] + 1) * (g.n[2] + 1);
  g.nface[0] = (g.n[0] + 1) * g.n[1] * g.n[2];
  g.nface[1] = g.n[0] * (g.n[1] + 1) * g.n[2];
  g.nface[2] = g.n[0] * g.n[1] * (g.n[2] + 1);
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 3; ++q) g.wu[a][s][q] = q == a ? 0.0 : 2.0 * urand() - 1.0;
  geom_finish(g);
  const size_t nc = g.ncell;
  const float beta = (float)(0.3 * g.h * g.h * (1.0 + 40.0 * urand()));
  std::vector<float> u(3 * nc), b(3 * nc), eta(nc);
  for (auto& v : u) v = (float)(2.0 * urand() - 1.0);
  for (auto& v : b) v = (float)(2.0 * urand() - 1.0);
  for (auto& v : eta) v = (float)(0.05 + 3.0 * urand());

  // the thread -> cell maps of the sweep (one colour) and of the operator
  // (both): every cell of a colour exactly once, the interior flag exactly on
  // the interior cells, P its position in the colour's half
  const SplitMap sm = split_map(g);
  const dim3 grid = split_grid(g);
  for (int ncol = 0; ncol <= 2; ++ncol)  // 0: the sweep's two-cell map
    for (int col0 = 0; col0 < (ncol < 2 ? 2 : 1); ++col0) {
      std::vector<int> seen(nc, 0);
      bool bad = false;
      auto visit = [&](const int* p, int P, int col, bool in) {
        if (p[0] < 0 || p[0] >= g.n[0] || p[1] < 0 || p[1] >= g.n[1] || p[2] < 0 || p[2] >= g.n[2] ||
            ((p[0] + p[1] + p[2]) & 1) != col || sidx(g, p[0], p[1], p[2]) != col * (g.ncell >> 1) + P ||
            in != interior<3>(g, p)) {
          bad = true;
          return;
        }
        ++seen[cidx<3>(g, p[0], p[1], p[2])];
      };
      auto visit2 = [&](const int* p, int P, bool in, bool ca, bool cb) {
        if (ca) visit(p, P, col0, in);
        if (cb) {
          const int p2[3] = {p[0] + 2, p[1], p[2]};
          visit(p2, P + 1, col0, in);
        }
      };
      const dim3 gr = ncol == 0 ? split_sweep_grid(g) : grid;
      const dim3 bl = ncol == 0 ? split_sweep_block(g) : split_block_dim(g, ncol);
      const int nt = (int)(bl.x * bl.y);
      for (int k = 0; k < (int)gr.z; ++k)
        for (int j = 0; j < (int)gr.y; ++j)
          for (int seg = 0; seg < (int)gr.x; ++seg)
            for (int tid = 0; tid < nt; ++tid) {
              if (ncol == 0)
                split_pair_thread(g, col0, split_sweep(g), seg, j, k, tid % (int)bl.x, tid / (int)bl.x, visit2);
              else if (ncol == 1)
                split_thread<1>(g, col0, sm.W, seg, j, k, tid, visit);
              else
                split_thread<2>(g, 0, sm.W, seg, j, k, tid, visit);
            }
      if (bad) return fail("a mapped cell (bounds, colour, position or interior flag)");
      for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j)
          for (int i = 0; i < g.n[0]; ++i) {
            const bool mine = ncol == 2 || ((i + j + k) & 1) == col0;
            if (seen[cidx<3>(g, i, j, k)] != (mine ? 1 : 0)) return fail("cell coverage");
          }
    }

  const std::vector<float> su0 = to_split(g, u, 3), sb = to_split(g, b, 3), seta = to_split(g, eta, 1);
  const CellEta<float> ce{eta.data()};

  // operator, without and with a right-hand side
  for (int withb = 0; withb < 2; ++withb) {
    std::vector<float> out(3 * nc, 0.f), sout(3 * nc, 0.f);
    const float* bp = withb ? b.data() : nullptr;
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i) {
          const int p[3] = {i, j, k};
          visc_op_cell<3, float, false>(u.data(), bp, out.data(), ce, g, beta, hom, p, cidx<3>(g, i, j, k));
        }
    for (int k = 0; k < (int)grid.z; ++k)
      for (int j = 0; j < (int)grid.y; ++j)
        for (int seg = 0; seg < (int)grid.x; ++seg)
          for (int tid = 0; tid < (int)split_block_dim(g, 2).x; ++tid)
            split_op_thread(su0.data(), withb ? sb.data() : nullptr, sout.data(), seta.data(), g, beta, hom, seg, j, k,
                            tid);
    if (!same_split(g, out, sout, 3)) return fail(withb ? "operator with b" : "operator");
  }

  // red-black sweeps of the three components in turn, by the scalar gather
  // and (rows of even length) by the 8-byte pair gather
  for (int vec = 0; vec < ((g.n[0] / 2) % 2 == 0 ? 2 : 1); ++vec) {
    std::vector<float> x = u, sx = su0;
    for (int C = 0; C < 3; ++C)
      for (int col = 0; col < 2; ++col) {
        for (int t = 0; t < rbx_count<3>(g); ++t) {
          int p[3];
          if (!rbx_cell<3>(g, t, col, p)) continue;
          if (C == 0) visc_smooth_cell<3, float, 0, false>(x.data(), b.data(), ce, g, beta, hom, p);
          if (C == 1) visc_smooth_cell<3, float, 1, false>(x.data(), b.data(), ce, g, beta, hom, p);
          if (C == 2) visc_smooth_cell<3, float, 2, false>(x.data(), b.data(), ce, g, beta, hom, p);
        }
        const dim3 sgr = split_sweep_grid(g), sbl = split_sweep_block(g);
        const SplitSweep sw = split_sweep(g);
        // the kernel rebuilds the map from its launch dimensions
        if ((int)sbl.x != sw.bx || (int)sbl.y != sw.R || (int)sgr.x != sw.nseg ||
            (int)sgr.y - (g.n[1] + 31) / 32 != sw.nb)
          return fail("sweep launch dimensions");
        for (int k = 0; k < (int)sgr.z; ++k)
          for (int j = 0; j < (int)sgr.y; ++j)
            for (int seg = 0; seg < (int)sgr.x; ++seg)
              for (int ty = 0; ty < (int)sbl.y; ++ty)
                for (int tx = 0; tx < (int)sbl.x; ++tx) {
                  if (C == 0 && vec) split_smooth_thread<0, true>(sx.data(), sb.data(), seta.data(), g, col, beta, hom, sw, seg, j, k, tx, ty);
                  if (C == 0 && !vec) split_smooth_thread<0, false>(sx.data(), sb.data(), seta.data(), g, col, beta, hom, sw, seg, j, k, tx, ty);
                  if (C == 1 && vec) split_smooth_thread<1, true>(sx.data(), sb.data(), seta.data(), g, col, beta, hom, sw, seg, j, k, tx, ty);
                  if (C == 1 && !vec) split_smooth_thread<1, false>(sx.data(), sb.data(), seta.data(), g, col, beta, hom, sw, seg, j, k, tx, ty);
                  if (C == 2 && vec) split_smooth_thread<2, true>(sx.data(), sb.data(), seta.data(), g, col, beta, hom, sw, seg, j, k, tx, ty);
                  if (C == 2 && !vec) split_smooth_thread<2, false>(sx.data(), sb.data(), seta.data(), g, col, beta, hom, sw, seg, j, k, tx, ty);
                }
        if (!same_split(g, x, sx, 3)) return fail(vec ? "red-black sweep (8-byte pairs)" : "red-black sweep");
      }
  }

  // conversions: out = (float)(a - bsub) and (float)a; x += sc d
  {
    std::vector<double> a(3 * nc), bsub(3 * nc), x(3 * nc);
    for (auto& v : a) v = 2.0 * urand() - 1.0;
    for (auto& v : bsub) v = 2.0 * urand() - 1.0;
    for (auto& v : x) v = 2.0 * urand() - 1.0;
    for (int withb = 0; withb < 2; ++withb) {
      std::vector<float> nat(3 * nc), spl(3 * nc);
      for (size_t t = 0; t < 3 * nc; ++t) nat[t] = withb ? (float)(a[t] - bsub[t]) : (float)a[t];
      for (long long tt = 0; tt < 3LL * (g.ncell >> 1); ++tt)
        split_from_pair(spl.data(), a.data(), withb ? bsub.data() : nullptr, g, tt);
      if (!same_split(g, nat, spl, 3)) return fail("conversion to the split layout");
    }
    const double sc = -0.37;
    std::vector<double> xn = x, xs = x;
    for (size_t t = 0; t < 3 * nc; ++t) xn[t] += sc * (double)u[t];
    for (long long tt = 0; tt < 3LL * (g.ncell >> 1); ++tt) split_add_pair(xs.data(), sc, su0.data(), g, tt);
    if (std::memcmp(xn.data(), xs.data(), xn.size() * sizeof(double)) != 0) return fail("update from the split layout");
  }

  // transfers between the split level and the natural coarse level
  if (g.n[1] % 2 == 0 && g.n[2] % 2 == 0) {
    const Geom gc = coarse_of<3>(g);
    std::vector<float> rc(3 * gc.ncell), src(3 * gc.ncell);
    for (long long t = 0; t < 3LL * gc.ncell; ++t) {
      k_restrict_cells_at<3, float>(u.data(), rc.data(), g, gc, 3, t);
      k_restrict_cells_at<3, float, true>(su0.data(), src.data(), g, gc, 3, t);
    }
    if (std::memcmp(rc.data(), src.data(), rc.size() * sizeof(float)) != 0) return fail("restriction");
    std::vector<float> ec(3 * gc.ncell);
    for (auto& v : ec) v = (float)(2.0 * urand() - 1.0);
    std::vector<float> x = u, sx = su0;
    for (long long t = 0; t < 3LL * gc.ncell; ++t) {
      k_prolong_cells_add_c_at<3, float, false>(x.data(), ec.data(), g, gc, -1.f, t);
      k_prolong_cells_add_c_at<3, float, false, true>(sx.data(), ec.data(), g, gc, -1.f, t);
    }
    if (!same_split(g, x, sx, 3)) return fail("prolongation");
  }
  return 0;
}
