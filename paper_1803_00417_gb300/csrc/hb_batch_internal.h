// Host-side structures of the batched sweep (many independent cavities
// advanced together, one persistent launch per stage).
#pragma once
#include <string>
#include <vector>

#include "hb_batch.cuh"

namespace hb {
namespace batch {


// a work list: tiles over one element space, cavity-major, with each
// cavity's first tile index (first[ncav] = total)
struct List {
  Tile* d = nullptr;
  int n = 0;
  int* dfirst = nullptr;
  std::vector<int> first;
};

// element spaces of a level (counts per cavity; 0 when the cavity is not in
// the list's set)
enum Space { kCells = 0, kCellsD, kRb, kNodes, kFaces, kMc0, kSpaces = kMc0 + 8 };

// the settings of a cavity that its argument tables capture
struct Sig {
  Rheo rheo;
  double rho, f[3], dt;
  int pv;
  SolverCfg cfg;
  const double *u, *ustar, *p;
  int walls_version;
  double theta;
};

struct Solvers;  // device argument tables of the solvers (hb_batch.cu)

}  // namespace batch
}  // namespace hb

struct hbf_batch {
  int dim = 2;
  int ncav = 0;
  int precision = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<hbf_ctx*> cav;
  std::vector<double> dt;   // per cavity
  std::vector<int> nlev;    // per cavity
  int maxlev = 0;
  int tile = 2048;          // elements per tile
  int blocks_per_sm = 8;    // persistent grid = 152 * blocks_per_sm blocks at most
  int tail_cells = 4096;    // levels whose every cavity has at most this many cells run fused
  int tail_level = 0;       // first such level (maxlev: none), set by prepare
  // H[l]: cavities that have level l; A[l]: cavities for which level l is
  // not the coarsest (they smooth, restrict and prolong there)
  hb::batch::List H[hb::batch::kMaxLev][hb::batch::kSpaces];
  hb::batch::List A[hb::batch::kMaxLev][hb::batch::kSpaces];
  int max_tiles = 0;
  std::vector<void*> tables;   // device argument tables (rebuilt with the lists)
  std::vector<void*> lallocs;  // list storage
  std::vector<void*> allocs;   // fixed storage
  int* mask_all = nullptr;     // ones
  int* mask_act = nullptr;     // active cavities of the running solve
  int* h_act = nullptr;        // pinned host copy
  std::vector<int> act_uploaded;
  bool h2d_pending = false;    // an upload from h_act / hscal may still be in flight
  double* part = nullptr;      // per tile partials
  double* red = nullptr;       // per cavity results, kRedSlots x ncav
  double* hred = nullptr;      // pinned host copy
  double* scal = nullptr;      // per cavity scalars of the vector updates, 4 x ncav
  double* hscal = nullptr;     // pinned host copy
  void* expl = nullptr;        // explicit-stage tables (hb_batch_explicit.cu)
  hb::batch::Solvers* sol = nullptr;
  bool prepared = false;
  std::vector<hb::batch::Sig> sig;
  long long nlaunch = 0;
  // phase timing (hbf_batch_profile): events between the stages of a step
  bool prof = false;
  cudaEvent_t pev[8] = {};
  double phase_ms[7] = {};
  long long prof_steps = 0;
  long long trips[3] = {};     // batched iterations of the MAC, viscous and nodal loops
  std::string err;
};

namespace hb {
namespace batch {
constexpr int kRedSlots = 4;

// explicit stages (hb_batch_explicit.cu): tables over the H[0] lists
void* explicit_create(hbf_batch* B);
void explicit_destroy(void* e);
// which: 0 eta, face eta, G p; 1 slopes, transverse terms, traces, MAC rhs;
// 2 MAC correction, advective rhs; 3 G p, nodal rhs; 4 projection update of u*
void explicit_stage(hbf_batch* B, void* e, int which);

// persistent launch of Op over list L (skipped when empty)
template <class Op>
inline void run(hbf_batch* B, const void* tab, const List& L, const int* mask, int extra = 0) {
  if (L.n == 0) return;
  int grid = 152 * B->blocks_per_sm;
  if (grid > L.n) grid = L.n;
  k_batch<Op><<<grid, kThreads, 0, B->stream>>>((const typename Op::Arg*)tab, L.d, L.n, mask, extra);
  ++B->nlaunch;
}

// copy a host vector of arguments into a new device table owned by B
template <class ArgT>
inline void* upload_table(hbf_batch* B, const std::vector<ArgT>& h) {
  void* d = nullptr;
  if (cudaMalloc(&d, sizeof(ArgT) * h.size()) != cudaSuccess) return nullptr;
  cudaMemcpy(d, h.data(), sizeof(ArgT) * h.size(), cudaMemcpyHostToDevice);
  B->tables.push_back(d);
  return d;
}

}  // namespace batch
}  // namespace hb
