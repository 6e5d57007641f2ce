// Host build of the multigrid pieces' per-element device functions, driven by
// tests/test_host_multigrid.py: operators, one smoothing sweep and the grid
// transfers of the three solves on a seeded state, for comparison with the
// oracle's.  No GPU needed.
//
// input:  int32 d, n0, n1, n2, hom; float64 h, beta, wall_u[3][2][3];
//         eta (ncell), u (d ncell), bv (d ncell), x (ncell), bc (ncell),
//         xn (nnode), bn (nnode), ev (d ncell_c), ec (ncell_c), en (nnode_c)
// output: A u (d ncell); u after one viscous sweep (d ncell); bc - L x;
//         x after one cell sweep; bn - L xn; xn after one nodal sweep;
//         restricted u (d ncell_c); coarse faces (sum of nface_c);
//         u + P ev (odd ghosts, d ncell); x + P ec (even ghosts);
//         restricted xn (nnode_c); xn + P en (nnode); then in FP32 with
//         the finest-level maps and cell viscosity: A u (d ncell) and u after
//         one viscous sweep (d ncell); x after one FP32 cell sweep; xn after
//         one FP32 nodal sweep; all written as float64
#include <cstdio>
#include <cstring>
#include <vector>

#include "hb_internal.h"
#include "hb_mg_kernels.cuh"

using namespace hb;

template <typename T>
static bool rd(FILE* f, std::vector<T>& v) {
  return std::fread(v.data(), sizeof(T), v.size(), f) == v.size();
}

template <typename T>
static void wr(FILE* f, const std::vector<T>& v) {
  std::fwrite(v.data(), sizeof(T), v.size(), f);
}

template <int D, int C>
static void visc_colour_sweep(std::vector<double>& u, const std::vector<double>& b, const double* const* ef,
                              const Geom& g, double beta, int hom) {
  for (int col = 0; col < 2; ++col)
    for (int t = 0; t < rb_count<D>(g); ++t)
      k_visc_smooth_c_at<D, double, C>(u.data(), b.data(), ef[0], ef[1], ef[2], g, col, beta, hom, t);
}

template <int D, int C>
static void fsweep(std::vector<float>& u, const std::vector<float>& b, const CellEta<float>& ce, const Geom& g,
                   float beta, int hom) {
  for (int col = 0; col < 2; ++col)
    for (int t = 0; t < rbx_count<D>(g); ++t) {
      int p[3];
      if (rbx_cell<D>(g, t, col, p)) visc_smooth_cell<D, float, C>(u.data(), b.data(), ce, g, beta, hom, p);
    }
}

template <int D>
static int run(FILE* in, FILE* out, const int* n, int hom) {
  std::vector<double> hd(2), wu(18);
  if (!rd(in, hd) || !rd(in, wu)) return 2;
  Geom g;
  std::memset(&g, 0, sizeof g);
  g.n[0] = n[0];
  g.n[1] = n[1];
  g.n[2] = D == 3 ? n[2] : 1;
  g.h = hd[0];
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  g.nnode = (g.n[0] + 1) * (g.n[1] + 1) * (D == 3 ? g.n[2] + 1 : 1);
  g.nface[0] = (g.n[0] + 1) * g.n[1] * g.n[2];
  g.nface[1] = g.n[0] * (g.n[1] + 1) * g.n[2];
  g.nface[2] = D == 3 ? g.n[0] * g.n[1] * (g.n[2] + 1) : 0;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 3; ++q) g.wu[a][s][q] = wu[(a * 2 + s) * 3 + q];
  geom_finish(g);
  const Geom gc = coarse_of<D>(g);
  const double beta = hd[1];
  const size_t nc = g.ncell, nn = g.nnode, ncc = gc.ncell, nnc = gc.nnode;
  std::vector<double> eta(nc), u(D * nc), bv(D * nc), x(nc), bc(nc), xn(nn), bn(nn), ev(D * ncc), ec(ncc),
      en(nnc);
  if (!rd(in, eta) || !rd(in, u) || !rd(in, bv) || !rd(in, x) || !rd(in, bc) || !rd(in, xn) || !rd(in, bn) ||
      !rd(in, ev) || !rd(in, ec) || !rd(in, en))
    return 3;
  // level-0 faces by the finest-level rule
  std::vector<double> ef[3];
  const double* efp[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < D; ++a) {
    ef[a].resize(g.nface[a]);
    for (int t = 0; t < g.nface[a]; ++t) {
      int p[3];
      face_coords(g, a, t, p[0], p[1], p[2]);
      int L[3] = {p[0], p[1], p[2]}, R[3] = {p[0], p[1], p[2]};
      L[a] = p[a] > 0 ? p[a] - 1 : 0;
      R[a] = p[a] < g.n[a] ? p[a] : g.n[a] - 1;
      ef[a][t] = 0.5 * (eta[cidx<D>(g, L[0], L[1], L[2])] + eta[cidx<D>(g, R[0], R[1], R[2])]);
    }
    efp[a] = ef[a].data();
  }
  std::vector<double> Au(D * nc);
  for (int t = 0; t < g.ncell; ++t)
    k_visc_op_at<D, double>(u.data(), nullptr, Au.data(), efp[0], efp[1], efp[2], g, beta, hom, t);
  wr(out, Au);
  std::vector<double> us = u;
  visc_colour_sweep<D, 0>(us, bv, efp, g, beta, hom);
  visc_colour_sweep<D, 1>(us, bv, efp, g, beta, hom);
  if (D == 3) visc_colour_sweep<D, (D == 3 ? 2 : 0)>(us, bv, efp, g, beta, hom);
  wr(out, us);
  std::vector<double> r(nc);
  for (int t = 0; t < g.ncell; ++t) k_cell_resid_at<D, double>(x.data(), bc.data(), r.data(), g, t);
  wr(out, r);
  std::vector<double> xs = x;
  for (int col = 0; col < 2; ++col)
    for (int t = 0; t < rb_count<D>(g); ++t) k_cell_smooth_at<D, double>(xs.data(), bc.data(), g, col, t);
  wr(out, xs);
  std::vector<double> rn(nn);
  for (int t = 0; t < g.nnode; ++t) k_nodal_resid_at<D, double>(xn.data(), bn.data(), rn.data(), g, t);
  wr(out, rn);
  std::vector<double> xns = xn;
  for (int col = 0; col < (1 << D); ++col)
    for (int t = 0; t < mc_count<D>(g, col); ++t) k_nodal_smooth_at<D, double>(xns.data(), bn.data(), g, col, t);
  wr(out, xns);
  std::vector<double> ur(D * ncc);
  for (long long t = 0; t < (long long)D * gc.ncell; ++t) k_restrict_cells_at<D, double>(u.data(), ur.data(), g, gc, D, t);
  wr(out, ur);
  for (int a = 0; a < D; ++a) {
    std::vector<double> fc(gc.nface[a]);
    for (int t = 0; t < gc.nface[a]; ++t) k_restrict_faces_at<D, double>(efp[a], fc.data(), a, g, gc, t);
    wr(out, fc);
  }
  // prolongation: the coarse-centred form the level-by-level cycles launch,
  // checked bit for bit against the per-fine-cell form of the fused tail
  std::vector<double> up = u, up1 = u;
  for (long long t = 0; t < (long long)D * gc.ncell; ++t)
    k_prolong_cells_add_c_at<D, double>(up.data(), ev.data(), g, gc, -1.0, t);
  for (long long t = 0; t < (long long)D * g.ncell; ++t)
    k_prolong_cells_add_at<D, double>(up1.data(), ev.data(), g, gc, D, -1.0, t);
  if (std::memcmp(up.data(), up1.data(), up.size() * sizeof(double)) != 0) {
    std::fprintf(stderr, "the two cell prolongations differ (Dirichlet)\n");
    return 3;
  }
  wr(out, up);
  std::vector<double> xp = x, xp1 = x;
  for (long long t = 0; t < gc.ncell; ++t) k_prolong_cells_add_c_at<D, double>(xp.data(), ec.data(), g, gc, 1.0, t);
  for (long long t = 0; t < g.ncell; ++t) k_prolong_cells_add_at<D, double>(xp1.data(), ec.data(), g, gc, 1, 1.0, t);
  if (std::memcmp(xp.data(), xp1.data(), xp.size() * sizeof(double)) != 0) {
    std::fprintf(stderr, "the two cell prolongations differ (Neumann)\n");
    return 3;
  }
  wr(out, xp);
  std::vector<double> nr(nnc);
  for (int t = 0; t < gc.nnode; ++t) k_restrict_nodes_at<D, double>(xn.data(), nr.data(), g, gc, t);
  wr(out, nr);
  std::vector<double> np_ = xn;
  for (int t = 0; t < g.nnode; ++t) k_prolong_nodes_add_at<D, double>(np_.data(), en.data(), g, gc, t);
  wr(out, np_);
  // the FP32 finest level of the mixed V-cycles as its kernels walk it: the
  // x-interior-first maps, face viscosities formed from the cell viscosity
  std::vector<float> fu(u.begin(), u.end()), fb(bv.begin(), bv.end()), feta(eta.begin(), eta.end());
  std::vector<float> fAu(D * nc);
  const CellEta<float> ce{feta.data()};
  for (int t = 0; t < xi_count<D>(g); ++t) {
    int p[3];
    if (xi_cell<D>(g, t, p))
      visc_op_cell<D, float>(fu.data(), nullptr, fAu.data(), ce, g, (float)beta, hom, p, cidx<D>(g, p[0], p[1], p[2]));
  }
  wr(out, std::vector<double>(fAu.begin(), fAu.end()));
  fsweep<D, 0>(fu, fb, ce, g, (float)beta, hom);
  fsweep<D, 1>(fu, fb, ce, g, (float)beta, hom);
  if (D == 3) fsweep<D, (D == 3 ? 2 : 0)>(fu, fb, ce, g, (float)beta, hom);
  wr(out, std::vector<double>(fu.begin(), fu.end()));
  // the FP32 cell and nodal Poisson sweeps of the mixed MAC and nodal solves
  std::vector<float> fx(x.begin(), x.end()), fbc(bc.begin(), bc.end());
  for (int col = 0; col < 2; ++col)
    for (int t = 0; t < rb_count<D>(g); ++t) k_cell_smooth_at<D, float>(fx.data(), fbc.data(), g, col, t);
  wr(out, std::vector<double>(fx.begin(), fx.end()));
  std::vector<float> fxn(xn.begin(), xn.end()), fbn(bn.begin(), bn.end());
  for (int col = 0; col < (1 << D); ++col)
    for (int t = 0; t < mc_count<D>(g, col); ++t) k_nodal_smooth_at<D, float>(fxn.data(), fbn.data(), g, col, t);
  wr(out, std::vector<double>(fxn.begin(), fxn.end()));
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* in = std::fopen(argv[1], "rb");
  FILE* out = std::fopen(argv[2], "wb");
  if (!in || !out) return 1;
  int hd[5];
  if (std::fread(hd, sizeof(int), 5, in) != 5) return 2;
  const int n[3] = {hd[1], hd[2], hd[3]};
  const int st = hd[0] == 3 ? run<3>(in, out, n, hd[4]) : run<2>(in, out, n, hd[4]);
  std::fclose(in);
  std::fclose(out);
  return st;
}
