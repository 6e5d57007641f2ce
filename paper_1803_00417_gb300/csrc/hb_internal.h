// Host-side internals shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "hb_common.cuh"
#include "../../include/hbflow.h"

namespace hb {

struct Level {
  Geom g;
  // viscous solve (d components each)
  double* vx = nullptr;
  double* vb = nullptr;
  double* vr = nullptr;
  double* ef[3] = {nullptr, nullptr, nullptr};  // face eta
  // cell Poisson (MAC)
  double* cx = nullptr;
  double* cb = nullptr;
  double* cr = nullptr;
  // nodal Poisson
  double* nx = nullptr;
  double* nb = nullptr;
  double* nr = nullptr;
  // FP32 copies for the mixed-precision V-cycles
  float* fvx = nullptr;
  float* fvb = nullptr;
  float* fvr = nullptr;
  float* fef[3] = {nullptr, nullptr, nullptr};
  float* feta = nullptr;  // level 0: the cell viscosity, whose face means the FP32 kernels form
  float* fvx2 = nullptr;  // level 0 in 3D: the second array of the fused red-black sweeps
  float* fcx = nullptr;
  float* fcb = nullptr;
  float* fcr = nullptr;
  float* fnx = nullptr;
  float* fnb = nullptr;
  float* fnr = nullptr;
};

// profiling slots: device time of every launch of one kernel class on the
// finest level, recorded with CUDA events on the context stream
enum ProfSlot {
  kSlotViscSmooth = 0,
  kSlotViscResid = 1,
  kSlotNodalSmooth = 2,
  kSlotNodalResid = 3,
  kSlotCellSmooth = 4,
  kSlotCellResid = 5,
  kSlotExplicit = 6,
  // detail slots (recorded only at profiling level 2)
  kSlotBottom = 7,
  kSlotTransfer = 8,
  kSlotReduce = 9,
  kSlotVector = 10,
  kSlotCoarse = 11,
  // region slot (level 2): a whole learned-guess section, its launches
  // included (they are also counted in their own slots)
  kSlotGuess = 12,
  kSlotCount = 13,
  kSlotNone = -1
};

struct Prof {
  int level = 0;  // 0 off, 1 main slots, 2 main + detail slots
  std::vector<cudaEvent_t> ev[kSlotCount];  // start/stop pairs
  size_t used[kSlotCount] = {};
};

inline bool prof_wants(const Prof& P, int slot) {
  return slot >= 0 && P.level > 0 && (slot < kSlotBottom || P.level > 1);
}

constexpr size_t kProfPairs = 16384;

// exact coarsest-level solve: inverse of the (bordered, for singular
// problems) dense operator of the bottom level
constexpr int kDenseMax = 128;  // unknowns
struct Dense {
  double* Minv = nullptr;  // (kDenseMax+1)^2
  int n = 0;               // matrix size (unknowns, +1 when bordered)
  bool valid = false;
};

struct SolverCfg {
  double rtol = 1e-10;
  int max_cycles = 200;
  int nu1 = 2, nu2 = 2, nu_bottom = 40;
};

}  // namespace hb

struct hbf_ctx {
  int dim = 2;
  int precision = 0;
  cudaStream_t stream = nullptr;
  hb::Geom g;
  hb::Rheo rheo;
  double rho = 1.0;
  double f[3] = {0, 0, 0};
  int predictor_visc = 0;
  int fused_sweep = 0;      // FP32 finest-level viscous sweeps in one launch per component (3D)
  int staged_tx = 0;        // FP32 finest-level viscous sweeps staged by TMA: tile width 64 or 128, 0 off (3D)
  int staged_tz = 16;       // planes per block of the staged sweeps
  int staged_op_rows = 0;   // FP32 finest-level viscous operator staged by TMA: tile 64 x 4 or 64 x 8, 0 off (3D)
  int staged_op_tz = 16;    // planes per block of the staged operator
  int* sweep_err = nullptr; // set by a staged sweep whose bounded wait gave up
  double K = 1.0;           // the consistency K as given to hbf_set_rheology
  double theta = 0.5;       // implicit weight of the viscous term (1/2: Crank-Nicolson, Eq. 15)
  double inner_drop = 1e-3; // residual drop of each FP32 BiCGStab pass of the mixed viscous solve
  int split_layout = 1;     // FP32 finest level of the mixed viscous solve in the colour-split layout where it applies
  int split_last = -1;      // the layout of the last mixed viscous solve (vprev32 is kept in it)
  double t = 0.0;           // time: the sum of the dt of every step taken
  long long nstep = 0;      // steps taken
  int walls_version = 0;    // bumped by hbf_set_walls (batched tables rebuild)
  bool prev_valid = false;  // ustar holds u^m of the last hbf_step (hbf_step_change)
  // diagnostics scratch, allocated on first use: d*ncell doubles, 2*ncell ints
  double* dscr = nullptr;
  int* dlab = nullptr;
  unsigned long long* dcnt = nullptr;  // 8 counters
  hb::SolverCfg cfg;
  std::string err;

  // fields (device)
  double* u = nullptr;      // d*ncell
  double* p = nullptr;      // nnode
  double* eta = nullptr;    // ncell
  double* ustar = nullptr;  // d*ncell
  double* rhs = nullptr;    // d*ncell
  double* Gp = nullptr;     // d*ncell
  double* Lu = nullptr;     // d*ncell
  double* slopes = nullptr; // d*d*ncell  [a][c]
  double* hats = nullptr;   // d*d*ncell  [b][c]
  double* tcom = nullptr;
  double* wn = nullptr;     // d*ncell: u*/dt + G p/rho, the nodal divergence's cell field   // d*d*ncell  [a][c]: the cell's share of the a-face traces
  double* uL[3] = {nullptr, nullptr, nullptr};   // per axis: d*nface[a]
  double* uR[3] = {nullptr, nullptr, nullptr};
  double* uadv[3] = {nullptr, nullptr, nullptr}; // per axis: nface[a]
  double* umac[3] = {nullptr, nullptr, nullptr};
  double* phi_mac = nullptr;  // ncell
  double* mrhs = nullptr;     // ncell, MAC right-hand side
  double* nrhs = nullptr;     // nnode
  double* nres0 = nullptr;    // nnode: warm-start residual of the last nodal solve
  // initial guess of the viscous solve (mixed precision): 0 u^m; 1 also a
  // minimal-residual step along the previous step's increment; 2 also one
  // along the learned network's direction
  int vguess_mode = 0;
  float* vprev32 = nullptr;   // d*ncell: u*^{m-1} - u^{m-1} of the last hbf_step
  bool vprev_ok = false;
  hbf_unet* vnet = nullptr;   // network of mode 2 and the level it runs on
  int vnet_level = 0;
  float* vnet_x = nullptr;
  int vrecord = 0;            // keep the solve's starting residual and correction
  double* vres0 = nullptr;    // d*ncell: b - A x at the start of the last solve (after the guess)
  double* vcorr = nullptr;    // d*ncell: u* minus the starting point of the last solve
  // learned initial guess (optional)
  hbf_unet* guess = nullptr;
  int guess_level = 0;        // multigrid level whose nodes the network sees
  double* ntry = nullptr;     // nnode: network correction on the nodes
  double* nzero = nullptr;    // nnode zeros
  float* net_x = nullptr;     // network input, one value per network point
  // BiCGStab vectors of the viscous solve (d*ncell each)
  double *kb = nullptr, *kr = nullptr, *krh = nullptr, *kp = nullptr, *kv = nullptr, *ks = nullptr,
         *kt = nullptr, *kph = nullptr, *ksh = nullptr;
  // FP32 BiCGStab vectors of the mixed-precision viscous solve
  float *fkr = nullptr, *fkrh = nullptr, *fkp = nullptr, *fkv = nullptr, *fks = nullptr, *fkt = nullptr,
        *fkph = nullptr, *fksh = nullptr, *fke = nullptr;
  // reductions
  double* partial = nullptr;  // 2 kRedBlocks doubles
  double* dres = nullptr;     // device result slot(s)
  double* hres = nullptr;     // pinned host result
  std::vector<hb::Level> lv;
  std::vector<void*> allocs;
  hb::Prof prof;
  long long nlaunch = 0;
  hb::Dense dense[3];  // viscous, MAC, nodal
  // fused V-cycle tail of the solves: levels >= tail_lf run in one block
  int tail_lf = -1;                         // -1: not set up; >= levels: none
  int tail_cells = 512;                     // the tail starts at the first level with at most this many cells
  void* tail_dev[3][2] = {};                // device argument records [kind][FP32?]
  std::vector<unsigned char> tail_host[3][2];
  double tail_beta[2] = {0.0, 0.0};         // beta of the uploaded viscous records
  double *dX = nullptr, *dM = nullptr, *dA = nullptr;  // build scratch
};

namespace hb {

constexpr int kRedBlocks = 1024;

// beta = theta dt / rho of the viscous solve; theta = 1/2 is computed as
// dt / (2 rho), the Crank-Nicolson form of Eq. 15
inline double visc_beta(double dt, double rho, double theta) {
  return theta == 0.5 ? dt / (2.0 * rho) : theta * dt / rho;
}

void prof_mark(hbf_ctx* c, int slot, bool start);

// brackets a whole section with one pair of events of a region slot
struct ProfRegion {
  hbf_ctx* c;
  int slot;
  bool on;
  ProfRegion(hbf_ctx* ctx, int s);
  ~ProfRegion();
};

// every kernel launch of the library goes through here: counts it and, when
// profiling is on, brackets finest-level launches of a slot with events
template <typename K, typename... Args>
inline void launch(hbf_ctx* c, int slot, K kern, int grid, int block, Args... args) {
  const bool rec = prof_wants(c->prof, slot);
  if (rec) prof_mark(c, slot, true);
  kern<<<grid, block, 0, c->stream>>>(args...);
  if (rec) prof_mark(c, slot, false);
  ++c->nlaunch;
}

template <typename K, typename... Args>
inline void launch3(hbf_ctx* c, int slot, K kern, dim3 grid, dim3 block, Args... args) {
  const bool rec = prof_wants(c->prof, slot);
  if (rec) prof_mark(c, slot, true);
  kern<<<grid, block, 0, c->stream>>>(args...);
  if (rec) prof_mark(c, slot, false);
  ++c->nlaunch;
}

template <typename K, typename... Args>
inline void launch_smem(hbf_ctx* c, int slot, K kern, dim3 grid, dim3 block, size_t smem, Args... args) {
  const bool rec = prof_wants(c->prof, slot);
  if (rec) prof_mark(c, slot, true);
  kern<<<grid, block, smem, c->stream>>>(args...);
  if (rec) prof_mark(c, slot, false);
  ++c->nlaunch;
}

// error helpers
int fail(hbf_ctx* c, int code, const std::string& msg);
int cuda_check(hbf_ctx* c, cudaError_t e, const char* what);

// explicit stages (hb_explicit.cu)
int launch_eta(hbf_ctx* c);
int launch_predict(hbf_ctx* c, double dt);
int launch_mac_rhs(hbf_ctx* c, double* rhs);
int launch_mac_correct(hbf_ctx* c, const double* phi);
int launch_advect_rhs(hbf_ctx* c, double dt);
int launch_nodal_rhs(hbf_ctx* c, double dt, const double* ustar, const double* p, double* out);
int launch_project_update(hbf_ctx* c, double dt, double* u, const double* p_old,
                          const double* phi);
int launch_eta_faces(hbf_ctx* c);

// reductions (hb_mg.cu)
double reduce_max_abs(hbf_ctx* c, const double* x, long long n, int* st);
double reduce_sum(hbf_ctx* c, const double* x, long long n, int* st);
double reduce_dot(hbf_ctx* c, const double* a, const double* b, long long n, int* st);

// solves (hb_mg.cu)
int solve_mac(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s);
int solve_viscous(hbf_ctx* c, double beta, const double* rhs, double* u, hbf_solve_stats* s);
int solve_nodal(hbf_ctx* c, const double* rhs, double* phi, hbf_solve_stats* s);
int nodal_residual(hbf_ctx* c, const double* b, const double* x, double* r);
// FP64 nodal full weighting from level l to l+1, and coarse += P fine correction
void nodal_restrict(hbf_ctx* c, int l, const double* fine, double* coarse);
void nodal_prolong_add(hbf_ctx* c, int l, double* fine, const double* coarse);
int tensor_lu(hbf_ctx* c, const double* u, double* out);  // out = L_eta u, finest level
bool ensure_dense(hbf_ctx* c, int kind, double beta);      // dense bottom inverse ready?
void axmy(hbf_ctx* c, double* out, const double* x, double a, const double* y, long long n);  // out = x - a y

// learned initial guess (hb_unet.cu): replaces p by the network's guess when
// that lowers the residual; *used tells which
int apply_guess(hbf_ctx* c, const double* b, double* p, int* used);
void release_guess(hbf_ctx* c);
void release_visc_guess(hbf_ctx* c);
int take_tc_err(hbf_unet* N, cudaStream_t s);
// the network's direction for the viscous residual r32 (FP32, d*ncell, finest
// level) scaled by `scale`, into d32 (FP32, d*ncell); false if none
bool visc_net_direction(hbf_ctx* c, const float* r32, double scale, float* d32);
// FP32 cell transfers of d-component fields between levels l and l + 1
void cell_restrict_f(hbf_ctx* c, int l, const float* fine, float* coarse);
void cell_restrict_d(hbf_ctx* c, int l, const double* fine, double* coarse, int ncomp);
void cell_prolong_add_f(hbf_ctx* c, int l, float* fine, const float* coarse);
// after a viscous solve of hbf_step: the increment for the next step's
// guess and the recorded correction
int visc_after_solve(hbf_ctx* c, const double* ustar, const double* u);

}  // namespace hb
