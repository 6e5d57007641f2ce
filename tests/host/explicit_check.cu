// Host build of the explicit-stage device functions (the same per-element code
// the kernels run), driven by tests/test_host_explicit.py: reads a seeded
// state, evaluates viscosity, face viscosities, G p, L_eta u, slopes,
// transverse terms, face states, u^adv and the nodal right-hand side, and
// writes them for comparison with the oracle.  No GPU needed.
//
// input:  int32 d, n0, n1, n2, pv; float64 h, dt, rho, K, nexp, tau_y, m,
//         f[3], wall_u[3][2][3]; u (d ncell), p (nnode), u* (d ncell)
// output: eta (ncell), Gp (d ncell), Lu (d ncell), then per axis a < d:
//         uL (d nface_a), uR (d nface_a), uadv (nface_a); nodal rhs (nnode)
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hb_internal.h"
#include "hb_explicit.cuh"
#include "hb_mg_kernels.cuh"

using namespace hb;

template <typename T>
static bool rd(FILE* f, T* v, size_t n) {
  return std::fread(v, sizeof(T), n, f) == n;
}

template <typename T>
static void wr(FILE* f, const std::vector<T>& v) {
  std::fwrite(v.data(), sizeof(T), v.size(), f);
}

template <int D>
static int run(FILE* in, FILE* out, const int* n, int pv) {
  double h, dt, rho, K, nexp, tau, m, fc[3], wu[18];
  if (!rd(in, &h, 1) || !rd(in, &dt, 1) || !rd(in, &rho, 1) || !rd(in, &K, 1) || !rd(in, &nexp, 1) ||
      !rd(in, &tau, 1) || !rd(in, &m, 1) || !rd(in, fc, 3) || !rd(in, wu, 18))
    return 2;
  Geom g;
  std::memset(&g, 0, sizeof g);
  g.n[0] = n[0];
  g.n[1] = n[1];
  g.n[2] = D == 3 ? n[2] : 1;
  g.h = h;
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  g.nnode = (g.n[0] + 1) * (g.n[1] + 1) * (D == 3 ? g.n[2] + 1 : 1);
  g.nface[0] = (g.n[0] + 1) * g.n[1] * g.n[2];
  g.nface[1] = g.n[0] * (g.n[1] + 1) * g.n[2];
  g.nface[2] = D == 3 ? g.n[0] * g.n[1] * (g.n[2] + 1) : 0;
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 3; ++q) g.wu[a][s][q] = wu[(a * 2 + s) * 3 + q];
  geom_finish(g);
  Rheo r;
  r.c2 = std::pow(2.0, nexp - 1.0) * K;
  r.n = nexp;
  r.tau = tau;
  r.m = m;
  r.reg_power = 1;
  r.e2 = rheo_e2(nexp, 1);
  const size_t nc = (size_t)g.ncell, nn = (size_t)g.nnode;
  std::vector<double> u(D * nc), p(nn), us(D * nc);
  if (!rd(in, u.data(), u.size()) || !rd(in, p.data(), nn) || !rd(in, us.data(), us.size())) return 3;

  std::vector<double> eta(nc), ef[3], Gp(D * nc), Lu(D * nc), slopes(D * D * nc), hats(D * D * nc),
      tcom(D * D * nc), w(D * nc), Gp2(D * nc), nrhs(nn);
  for (int t = 0; t < g.ncell; ++t) k_eta_at<D>(u.data(), eta.data(), g, r, t);
  for (int a = 0; a < D; ++a) {
    ef[a].resize(g.nface[a]);
    for (int t = 0; t < g.nface[a]; ++t) k_eta_faces_at<D>(eta.data(), ef[a].data(), a, g, t);
  }
  const double* e2 = D == 3 ? ef[2].data() : nullptr;
  for (int t = 0; t < g.ncell; ++t) k_grad_p_at<D>(p.data(), Gp.data(), g, t);
  for (int t = 0; t < g.ncell; ++t)
    k_tensor_lu_at<D, double>(u.data(), Lu.data(), ef[0].data(), ef[1].data(), e2, g, 0, t);
  for (int t = 0; t < g.ncell; ++t) k_slopes_at<D>(u.data(), slopes.data(), g, t);
  const StepC k = step_consts(g, D, dt, rho);
  const Force fo{{fc[0], fc[1], fc[2]}};
  for (int t = 0; t < g.ncell; ++t)
    k_hats_at<D>(u.data(), slopes.data(), Gp.data(), Lu.data(), fo, pv, hats.data(), tcom.data(), g, k, t);
  wr(out, eta);
  wr(out, Gp);
  wr(out, Lu);
  for (int a = 0; a < D; ++a) {
    std::vector<double> uL((size_t)D * g.nface[a]), uR((size_t)D * g.nface[a]), ua(g.nface[a]);
    for (int t = 0; t < g.nface[a]; ++t)
      k_traces_at<D>(u.data(), slopes.data(), tcom.data(), a, uL.data(), uR.data(), ua.data(), g, k, t);
    wr(out, uL);
    wr(out, uR);
    wr(out, ua);
  }
  for (int t = 0; t < g.ncell; ++t) k_grad_p_w_at<D>(p.data(), us.data(), Gp2.data(), w.data(), g, k, t);
  for (int t = 0; t < g.nnode; ++t) k_nodal_rhs_at<D>(w.data(), nrhs.data(), g, k, t);
  wr(out, nrhs);
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* in = std::fopen(argv[1], "rb");
  FILE* out = std::fopen(argv[2], "wb");
  if (!in || !out) return 1;
  int hd[5];
  if (!rd(in, hd, 5)) return 2;
  const int n[3] = {hd[1], hd[2], hd[3]};
  const int st = hd[0] == 3 ? run<3>(in, out, n, hd[4]) : run<2>(in, out, n, hd[4]);
  std::fclose(in);
  std::fclose(out);
  return st;
}
