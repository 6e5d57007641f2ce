// Host-side checks of integer helpers shared by the CUDA kernels, built and
// run by tests/test_host_helpers.py (no GPU needed; the same functions run on
// the device with the hi/lo register intrinsics in place of memcpy):
//  * the FP64 sign tests, magnitude minimum, limiter clamp and exact x/2, 2x
//    on bit patterns against plain IEEE arithmetic, bit for bit;
//  * the thread -> cell maps that put x-wall cells in warps of their own:
//    every cell (every cell of a red-black colour) exactly once, in range;
//  * the wall stencil of the viscous operator with its one-axis reflections
//    against the general reflection accessor, bit for bit;
//  * the interior smoother and operator (stored faces, and faces formed from
//    the cell viscosity) against the general point forms, and the cell-mean
//    face accessor against the finest-level face rule.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "hb_internal.h"
#include "hb_explicit.cuh"
#include "hb_fp64bits.cuh"
#include "hb_mg_kernels.cuh"

using namespace hb;

static uint64_t bits(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
}

static int fails = 0;
static void expect(bool ok, const char* what, double a, double b) {
  if (!ok && fails++ < 20) std::printf("FAIL %s a=%a b=%a\n", what, a, b);
}

static double sample(std::mt19937_64& rng) {
  std::uniform_int_distribution<int> kind(0, 9);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::uniform_int_distribution<uint64_t> any;
  switch (kind(rng)) {
    case 0: return 0.0;
    case 1: return -0.0;
    case 2: {  // subnormal
      uint64_t b = any(rng) & 0x000fffffffffffffull;
      if (any(rng) & 1) b |= 1ull << 63;
      double x;
      std::memcpy(&x, &b, 8);
      return x;
    }
    case 3: return std::ldexp(nd(rng), -1022 + (int)(any(rng) % 3));  // around the normal boundary
    case 4: return std::ldexp(nd(rng), 1020 + (int)(any(rng) % 4));   // near overflow
    case 5: return (any(rng) & 1) ? INFINITY : -INFINITY;
    case 6: {  // any finite pattern
      uint64_t b;
      double x;
      do {
        b = any(rng);
        std::memcpy(&x, &b, 8);
      } while (!std::isfinite(x));
      return x;
    }
    default: return nd(rng) * std::ldexp(1.0, (int)(any(rng) % 40) - 20);
  }
}

static void check_fp64bits() {
  std::mt19937_64 rng(12345);
  for (int it = 0; it < 2000000; ++it) {
    const double a = sample(rng), b = (it & 7) == 0 ? a : ((it & 7) == 1 ? -a : sample(rng));
    expect(dzero(a) == (a == 0.0), "dzero", a, 0);
    expect(dpos(a) == (a > 0.0), "dpos", a, 0);
    expect(dneg(a) == (a < 0.0), "dneg", a, 0);
    expect(bits(dhalf(a)) == bits(a * 0.5), "dhalf", a, 0);
    expect(bits(dtwice(a)) == bits(a * 2.0), "dtwice", a, 0);
    if (std::isfinite(a) && std::isfinite(b)) {
      expect(bits(dminabs(a, b)) == bits(std::fmin(std::fabs(a), std::fabs(b))), "dminabs", a, b);
      const double p = a * b;
      if (!(p == 0.0 && a != 0.0 && b != 0.0))  // the product underflowed
        expect(dsame_sign(a, b) == (p > 0.0), "dsame_sign", a, b);
      const double lim = std::fabs(b);
      double want;
      if (a == 0.0) {
        want = 0.0;
      } else {
        const double m = std::fmin(std::fabs(a), lim);
        want = a > 0.0 ? m : -m;
      }
      expect(bits(dsgn_min(a, lim)) == bits(want), "dsgn_min", a, lim);
    }
  }
}

template <int D>
static void check_maps(int n0, int n1, int n2) {
  Geom g{};
  g.n[0] = n0;
  g.n[1] = n1;
  g.n[2] = D == 3 ? n2 : 1;
  g.h = 1.0;
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  geom_finish(g);
  auto inside = [&](const int* p) {
    return p[0] >= 0 && p[0] < g.n[0] && p[1] >= 0 && p[1] < g.n[1] && p[2] >= 0 && p[2] < g.n[2];
  };
  for (int col = 0; col < 2; ++col) {
    std::vector<int> seen(g.ncell, 0);
    for (int t = 0; t < rbx_count<D>(g); ++t) {
      int p[3];
      if (!rbx_cell<D>(g, t, col, p)) continue;
      expect(inside(p), "rbx_cell range", n0, n1);
      if (inside(p)) seen[cidx<D>(g, p[0], p[1], p[2])]++;
    }
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i)
          expect(seen[cidx<D>(g, i, j, k)] == (((i + j + k + col) & 1) == 0 ? 1 : 0), "rbx_cell colour", n0, n1);
  }
  std::vector<int> seen(g.ncell, 0);
  for (int t = 0; t < xi_count<D>(g); ++t) {
    int p[3];
    if (!xi_cell<D>(g, t, p)) continue;
    expect(inside(p), "xi_cell range", n0, n1);
    if (inside(p)) seen[cidx<D>(g, p[0], p[1], p[2])]++;
  }
  for (int c = 0; c < g.ncell; ++c) expect(seen[c] == 1, "xi_cell once", n0, n1);
}

// the wall stencil's pieces against the same formulas with the general
// reflection accessor uget (every axis tested), bit for bit
template <int D, typename T>
static T ref_face_cross(const T* ua, const Geom& g, int a, int c, const int* L, bool hom) {
  if (L[a] < 0 || L[a] >= g.n[a] - 1) return T(0);
  int p1[3] = {L[0], L[1], L[2]}, p0[3] = {L[0], L[1], L[2]};
  p1[c] += 1;
  p0[c] -= 1;
  T dL = uget<D>(ua, g, a, p1[0], p1[1], p1[2], hom) - uget<D>(ua, g, a, p0[0], p0[1], p0[2], hom);
  p1[a] += 1;
  p0[a] += 1;
  T dR = uget<D>(ua, g, a, p1[0], p1[1], p1[2], hom) - uget<D>(ua, g, a, p0[0], p0[1], p0[2], hom);
  return (dL + dR) * g_q4<T>(g);
}

template <int D, typename T>
static T ref_tensor_point(const T* u, const T* const* ef, const Geom& g, int c, const int* p, bool hom) {
  const T* uc = u + (size_t)c * g.ncell;
  T acc = T(0);
  const T ih = g_ih<T>(g);
  for (int a = 0; a < D; ++a) {
    T flux[2];
    for (int s = 0; s < 2; ++s) {
      int L[3] = {p[0], p[1], p[2]};
      L[a] += s - 1;
      int R[3] = {L[0], L[1], L[2]};
      R[a] += 1;
      T e = ef[a][fidx(g, a, R[0], R[1], R[2])];
      T nrm = (uget<D>(uc, g, c, R[0], R[1], R[2], hom) - uget<D>(uc, g, c, L[0], L[1], L[2], hom)) * ih;
      if (a == c)
        flux[s] = e * (T(2) * nrm);
      else
        flux[s] = e * (nrm + ref_face_cross<D, T>(u + (size_t)a * g.ncell, g, a, c, L, hom));
    }
    acc += (flux[1] - flux[0]) * ih;
  }
  return acc;
}

template <int D, typename T>
static void check_wall_stencil(int n0, int n1, int n2) {
  Geom g{};
  g.n[0] = n0;
  g.n[1] = n1;
  g.n[2] = D == 3 ? n2 : 1;
  g.h = 1.0 / 7.0;
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  for (int a = 0; a < 3; ++a) g.nface[a] = (g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2 && D == 3));
  std::mt19937_64 rng(7 + n0 + 10 * n1 + 100 * n2);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd)
      for (int q = 0; q < 3; ++q) g.wu[a][sd][q] = nd(rng);
  geom_finish(g);
  std::vector<T> u((size_t)D * g.ncell), e[3];
  for (auto& v : u) v = (T)nd(rng);
  const T* ef[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < D; ++a) {
    e[a].resize(g.nface[a]);
    for (auto& v : e[a]) v = (T)(1.0 + std::fabs(nd(rng)));
    ef[a] = e[a].data();
  }
  for (int hom = 0; hom < 2; ++hom)
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i) {
          const int p[3] = {i, j, k};
          for (int c = 0; c < D; ++c) {
            const T got = mg_tensor_point<D, T>(u.data(), FaceEta<T>{ef}, g, c, p, hom != 0);
            const T want = ref_tensor_point<D, T>(u.data(), ef, g, c, p, hom != 0);
            expect(std::memcmp(&got, &want, sizeof(T)) == 0, "mg_tensor_point", (double)got, (double)want);
            for (int a = 0; a < D; ++a) {
              if (a == c) continue;
              for (int s = 0; s < 2; ++s) {
                int L[3] = {i, j, k};
                L[a] -= s;
                const T* ua = u.data() + (size_t)a * g.ncell;
                const T x = mg_face_cross<D, T>(ua, g, a, c, L, hom != 0);
                const T y = ref_face_cross<D, T>(ua, g, a, c, L, hom != 0);
                expect(std::memcmp(&x, &y, sizeof(T)) == 0, "mg_face_cross", (double)x, (double)y);
              }
            }
          }
        }
}

// the interior fast paths against the general (wall-aware) point forms on
// interior cells, with stored faces and with faces formed from cell
// viscosities; the cell-mean accessor against the finest-level face rule
template <int D>
static void check_interior_paths(int n0, int n1, int n2) {
  Geom g{};
  g.n[0] = n0;
  g.n[1] = n1;
  g.n[2] = D == 3 ? n2 : 1;
  g.h = 1.0 / 9.0;
  g.ncell = g.n[0] * g.n[1] * g.n[2];
  for (int a = 0; a < 3; ++a) g.nface[a] = (g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2 && D == 3));
  geom_finish(g);
  std::mt19937_64 rng(11 + n0 + 10 * n1 + 100 * n2);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<double> u((size_t)D * g.ncell), b((size_t)D * g.ncell), eta(g.ncell), e[3];
  for (auto& v : u) v = nd(rng);
  for (auto& v : b) v = nd(rng);
  for (auto& v : eta) v = std::exp(2.0 * nd(rng));
  const double* ef[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < D; ++a) {
    e[a].resize(g.nface[a]);
    for (int t = 0; t < g.nface[a]; ++t) k_eta_faces_at<D>(eta.data(), e[a].data(), a, g, t);
    ef[a] = e[a].data();
  }
  const FaceEta<double> fa{ef};
  const CellEta<double> ce{eta.data()};
  const Strides S = make_strides(g);
  const double beta = 0.37;
  auto close = [](double x, double y) { return std::fabs(x - y) <= 1e-12 * (1.0 + std::fabs(y)); };
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const int p[3] = {i, j, k};
        // every face through both accessors
        for (int a = 0; a < D; ++a)
          for (int s = 0; s < 2; ++s) {
            int q[3] = {i, j, k};
            q[a] += s;
            expect(fa.at(g, a, q) == ce.at(g, a, q), "CellEta::at", fa.at(g, a, q), ce.at(g, a, q));
          }
        if (!interior<D>(g, p)) continue;
        const int id = cidx<D>(g, i, j, k);
        for (int a = 0; a < D; ++a) {
          expect(CellEta<double>::kScale * ce.lo(g, S, a, p, id) == fa.lo(g, S, a, p, id), "CellEta::lo", 0, 0);
          expect(CellEta<double>::kScale * ce.hi(g, S, a, p, id) == fa.hi(g, S, a, p, id), "CellEta::hi", 0, 0);
        }
        for (int c = 0; c < D; ++c) {
          for (int hom = 0; hom < 2; ++hom) {
            const double w = visc_gs_point<D, double>(u.data(), b.data(), fa, g, c, p, beta, hom != 0);
            expect(close(visc_gs_interior<D, double>(u.data(), b.data(), fa, g, S, c, p, beta), w), "gs faces", w, 0);
            expect(close(visc_gs_interior<D, double>(u.data(), b.data(), ce, g, S, c, p, beta), w), "gs cells", w, 0);
            const double l = mg_tensor_point<D, double>(u.data(), fa, g, c, p, hom != 0);
            expect(close(tensor_interior<D, double>(u.data(), fa, g, S, c, p), l), "L faces", l, 0);
            expect(close(tensor_interior<D, double>(u.data(), ce, g, S, c, p), l), "L cells", l, 0);
          }
        }
      }
}

int main() {
  check_fp64bits();
  check_interior_paths<2>(7, 5, 1);
  check_interior_paths<3>(6, 5, 4);
  check_interior_paths<3>(3, 3, 3);
  for (int a : {1, 2, 3, 5})
    for (int b : {1, 2, 4}) {
      check_wall_stencil<2, double>(a, b, 1);
      check_wall_stencil<2, float>(a, b, 1);
      for (int c : {1, 3}) {
        check_wall_stencil<3, double>(a, b, c);
        check_wall_stencil<3, float>(a, b, c);
      }
    }
  const int sizes[] = {1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 33, 64};
  for (int a : sizes)
    for (int b : sizes) check_maps<2>(a, b, 1);
  for (int a : sizes)
    for (int b : {1, 2, 3, 8, 9})
      for (int c : {1, 2, 5, 8}) check_maps<3>(a, b, c);
  check_maps<3>(256, 256, 3);
  std::printf("%s (%d failures)\n", fails ? "FAILED" : "ok", fails);
  return fails ? 1 : 0;
}
