// Declarations shared by the translation units of the droplet library.
#pragma once
#include "common.cuh"
#include "adjoint_ad.cuh"

#include <vector>

namespace dg {

// launches issued by the library in this process
extern long long g_launches;

enum { KC_MG_SMOOTH = 0, KC_SPMV, KC_UPDATE, KC_MG_RESTRICT, KC_MG_PROLONG, KC_MOM_ASSEMBLE, KC_SCALAR_ASSEMBLE,
       KC_PCG_PERSIST, KC_COUNT };

// Optional CUDA-event timing of the kernel classes above (per context).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kind;        // kernel class of each recorded pair
  size_t used = 0;              // event pairs in use
  double bytes[KC_COUNT] = {0};
  double flops[KC_COUNT] = {0};   // algorithmic FP64 flops (0 for FP32 launches)
  long long n[KC_COUNT] = {0};
  int begin(int k, cudaStream_t st, double b, double f64 = 0.0);
  void end(int idx, cudaStream_t st);
  void reset();
  int read(int k, double* ms, long long* launches, double* bytes_total, double* flops_total = nullptr);
  void destroy();
};

struct ProfScope {
  Prof* p;
  cudaStream_t st;
  int idx;
  ProfScope(Prof* p_, int k, cudaStream_t st_, double b, double f64 = 0.0) : p(p_), st(st_), idx(-1) {
    if (p && p->on) idx = p->begin(k, st, b, f64);
  }
  ~ProfScope() {
    if (idx >= 0) p->end(idx, st);
  }
};

// indices of the per-droplet device scalar array
enum {
  SC_K = 0, SC_CLIP, SC_VAPOUT, SC_DT, SC_IDT, SC_TIME,
  SC_SUM_ALPHA_V, SC_SUM_MDOT_V, SC_SUM_TG, SC_SUM_G, SC_SUM_VAP, SC_SUM_MLIQ, SC_MAXU, SC_AMAX, SC_AMIN,
  SC_ITS_P, SC_ITS_T, SC_ITS_W, SC_ITS_U, SC_RES_P, SC_NC,
  SC_HIST,   // 1: the history fields hold the previous step's T, omega, u (extrapolated guesses)
  SC_COUNT
};

static_assert(SC_IDT == SC_DT + 1 && SC_TIME == SC_DT + 2, "the clock scalars are set together");

// dt and 1 / dt of the current step: the device scalars of a Courant-adaptive run (set by
// the diagnostics at the end of the previous step), else the configured constants
__device__ __forceinline__ double dt_of(const Phys& p) { return p.dyn ? p.dyn[SC_DT] : p.dt; }
__device__ __forceinline__ double idt_of(const Phys& p) { return p.dyn ? p.dyn[SC_IDT] : p.idt; }

// k_diag_finish modes: a state set from outside (dt and clock kept), the end of a step
// (clock advanced by the step's dt, the next dt from the Courant rule), an initial state
// (the first dt from the Courant rule, clock kept)
enum { DIAG_SET = 0, DIAG_STEP_END = 1, DIAG_INITIAL = 2 };

// ---- step kernels (step_kernels.cu)
__global__ void k_init(Geo g, Phys p, double* alpha, double* T, double* omega, double* rhoG);
__global__ void k_xi(Geo g, Phys p, double* xi);
__global__ void k_thermo_pin(Geo g, Phys p, const double* alpha, const double* T, double* omega,
                             const double* rhoG, double* rhoG_old, unsigned* flags, const int* dirty, double* scal);

__global__ void k_evap_K(const double* partials, int nblk, double* scal, unsigned* flags);
__global__ void k_alpha_source(Geo g, Phys p, const double* alpha, const double* mraw, const double* scal,
                               const double* T, const double* expand, double* mdot, double* alpha_star,
                               float* alpha_star_f, unsigned* flags, int* dirty);

__global__ void k_adv_low(Geo g, const double* as, const double* F0, const double* F1, const double* F2, double* aL);

__global__ void k_clip_finish(const double* partials, int nblk, double* scal, unsigned* flags);
// Binary32 copies of the stencil inputs of the mixed-precision assembly kernels (null
// pointers in FP64 runs): each element is f32_rn of its binary64 source, formed once
// where that value is formed (the S4 properties, with the step's old T and omega) or at
// the start of the step (the face velocities u^n), instead of once per stencil reference.
struct Shadow32 {
  float *T, *w;             // temperature and vapour mass fraction entering S5 / S6
  float *k, *gD;            // conductivity and rho D of the cell
  float *mu;                // viscosity
  float *u[3];              // face velocities
};
// mixture properties of a cell (S4), formed where alpha^{n+1} is (the FCT update, the clip)
struct PropsOut {
  const double *rhoG, *omega, *T;
  double *rho, *mu, *kc, *cp, *D;
  Shadow32 s;               // binary32 copies to write (s.T null: none)
  const unsigned char* solid = nullptr;   // the fibre's cells (null: no fibre): k = D = 0 there
};
// u^n rounded to binary32 (faces of every active direction in one launch)
__global__ void k_faces_f32(const double* u0, const double* u1, const double* u2, float* f0, float* f1, float* f2,
                            long long n0, long long n1, long long n2);
__global__ void k_alpha_clip_only(Geo g, Phys p, const double* as, double* alpha, double* partials, PropsOut po);

__global__ void k_yeq(Geo g, Phys p, const double* T, const double* alpha, const double* omega, double* yq,
                      unsigned* flags);
__global__ void k_species_noflow(Geo g, const double* alpha_new, const double* yq, double* omega);
__global__ void k_rhoG(Geo g, Phys p, const double* T, const double* w, double* rhoG);

__global__ void k_add(long long n, double* y, const double* x);

__global__ void k_diag_finish(const double* psum, const double* pmax, int nblk, double* scal, int mode,
                              double co_hmin, double dt_max);
__global__ void k_extrap(long long n, double* x, double* xh, const double* scal);

// launch wrappers of the kernels templated on the active axes / face direction (step_kernels.cu)
void L_evap_raw(cudaStream_t st, int grid, Geo g, Phys p, const double* alpha, const double* omega, const double* rhoG, const double* T, const double* u0, const double* u1, const double* u2, double* mraw, int* adj, double* partials, unsigned* flags);
void L_adv_faces(cudaStream_t st, int grid, Geo g, Phys p, int a, const double* as, const double* ua, double* FL, double* AF);
void L_adv_limit(cudaStream_t st, int grid, Geo g, const double* as, const double* aL, const double* A0, const double* A1, const double* A2, double* Rp, double* Rm);
void L_geo_advect(cudaStream_t st, int grid, Geo g, Phys p, const double* astar, double* const w[2],
                  double* const N[3], double* B, double* const u[3], double* alpha, double* partials, PropsOut po);
void L_adv_update(cudaStream_t st, int grid, Geo g, Phys p, const double* aL, const double* A0, const double* A1, const double* A2, const double* Rp, const double* Rm, double* alpha, double* partials, unsigned* flags, PropsOut po);
void L_scalar_assemble(cudaStream_t st, int grid, Geo g, Phys p, int mode, const double* phi, const double* rho, const double* cp, const double* kc, const double* D, const double* mdot, const double* u0, const double* u1, const double* u2, const double* alpha_new, const double* pinv, double amb, double* Dg, double* c0, double* c1, double* c2, double* rhs, const Shadow32* s32,
                       const double* wq = nullptr);
// the alpha face fluxes of every direction in one launch (mixed precision)
void L_adv_faces_mx_all(cudaStream_t st, Geo g, Phys p, const double* as, const float* asf, double* const u[3],
                        double* const FL[3], double* const AF[3]);
void L_scalar_assemble_mx(cudaStream_t st, int grid, Geo g, Phys p, int mode, const double* phi, const double* rho, const double* cp, const double* kc, const double* D, const double* mdot, const double* u0, const double* u1, const double* u2, const double* alpha_new, const double* pinv, double amb, double* Dg, double* c0, double* c1, double* c2, double* rhs, const Shadow32* s32,
                          const double* wq = nullptr);
void L_mom_assemble_mx(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* u0, const double* u1, const double* u2, const double* rho, const double* mu, const double* pr, const double* alpha, const double* xi, double* Dg, double* c0, double* c1, double* c2, double* rhs, const Shadow32* s32);
void L_mom_assemble(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* u0, const double* u1, const double* u2, const double* rho, const double* mu, const double* pr, const double* alpha, const double* xi, double* Dg, double* c0, double* c1, double* c2, double* rhs, const Shadow32* s32);
void L_mom_scatter(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* x, double* us);
void L_poisson_assemble(cudaStream_t st, int grid, Geo g, Phys p, const double* mdot, const double* alpha, const double* rgo, const double* rgn, const double* u0, const double* u1, const double* u2, const double* us0, const double* us1, const double* us2, const double* rho, const double* T1, const double* T0, double* expand, double* S, double* Dg, double* c0, double* c1, double* c2, double* rhs, double* dp0);
void L_correct(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* us, const double* dp, const double* rho, double* u);
// the velocity correction of every direction and p_rgh += dp in one launch
void L_correct_all(cudaStream_t st, Geo g, Phys p, double* const us[3], const double* dp, const double* rho,
                   double* const u[3], double* pr);
void L_diag(cudaStream_t st, int grid, Geo g, Phys p, const double* alpha, const double* T, const double* mdot, const double* omega, const double* rhoG, const double* u0, const double* u1, const double* u2, double* psum, double* pmax, unsigned* flags);

void L_faces_to_box(cudaStream_t st, int grid, const Geo& g, int c, const double* u, double* x, double* uh,
                    const double* scal);

// ---- adjoint of the step without flow (adjoint.cu)
// accumulators: gas diffusivity, J, ambient temperature through the initial field, and
// through the boundary values of the energy equation (flow only)
enum { AC_DGAS = 0, AC_J, AC_TAMB, AC_TAMB_BC, AC_COUNT };
void L_adj_pin(cudaStream_t st, const Geo& g, const Phys& p, const double* alpha, const double* T,
               const double* omega, double* wp);
void L_adj_rhs(cudaStream_t st, const Geo& g, const double* abar, const double* alpha_new, int pinned_rows,
               double* rhs, double* x);
void L_adj_species(cudaStream_t st, const Geo& g, const Phys& p, const double* bW, const double* aW, const double* aT,
                   const double* alpha_new, const double* wp, const double* wn1, const double* Tn1, const double* rho,
                   const double* D, double* Tn1bar, double* wpbar, double* rhobar, double* Dbar);
void L_adj_energy(cudaStream_t st, const Geo& g, const Phys& p, const double* bT, const double* Tn, const double* Tn1,
                  const double* rho, const double* cp, const double* kc, double* Tnbar, double* rhobar, double* kbar,
                  double* cpbar, double* mdbar);
void L_adj_source(cudaStream_t st, const Geo& g, const Phys& p, const double* aA, const double* alpha_n,
                  const double* alpha_new, const double* astar, const double* rgn, const double* mraw,
                  const double* scal, const double* rhobar, const double* kbar, const double* cpbar,
                  const double* Dbar, double jweight, double* aAn, double* rgbar, double* mdbar, double* mrbar,
                  double* part, double* acc_out);
void L_adj_evap(cudaStream_t st, const Geo& g, const Phys& p, const double* alpha_n, const double* wp,
                const double* rgn, const int* adj, const double* mrbar, double* aAn, double* wpbar, double* rgbar,
                double* part, double* acc_out);
void L_adj_thermo(cudaStream_t st, const Geo& g, const Phys& p, const double* alpha_n, const double* Tn,
                  const double* wp, const double* rgn, const double* rgbar, const double* wpbar, double* Tnbar,
                  double* aW);
void L_acc_J(cudaStream_t st, const double* scal, double weight, double* acc_out);
// K = S1/S2, mdot = K f m_raw: adjoint of m_raw and of alpha^n through f, from mdbar and the
// block sums {D_gas, mdbar f m_raw, m_raw V, f m_raw V} in part
void L_adj_K(cudaStream_t st, const Geo& g, const Phys& p, const double* part, int nblk, const double* alpha_n,
             const double* mraw, const double* scal, const double* mdbar, double* mrbar, double* aAn, double* acc_out);
void L_adj_tamb(cudaStream_t st, const Geo& g, const Phys& p, const double* T0bar, double* part, double* acc_out);

// ---- adjoint of the step with flow (adjoint_flow.cu)
// The forward step's state n and intermediates, as the adjoint reads them (the forward
// step n -> n+1 just re-run; u, p of state n kept aside)
struct FlowIn {
  const double *alpha_n, *T_n, *wp, *u[3], *p_n;
  const double *astar, *aL, *FL[3], *AF[3], *Rp, *Rm;
  const double *alpha1, *rho, *mu, *kc, *cp, *Dm, *mdot, *rgo, *rgn, *yq, *us[3], *dp, *xi;
  const int* adj;
};
// each launcher adds sum_j w_j d(out_j)/d(input) into the adjoints T of its inputs; the
// weights come from the arrays named (see adjoint_flow.cu)
void L_adjf_correct(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T,
                    double* const lU[3]);
void L_adjf_poisson(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, const double* mu,
                    const double* x);
void L_adjf_mom(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, int c,
                const double* mu, const double* x);
void L_adjf_scalar(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, int mode,
                   const double* mu, const double* x);
void L_adjf_fct(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T);
void L_adjf_mraw(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, const double* mrbar);
// box <-> faces of direction c: the interior faces' values into box order, and the adjoint
// of u* into the box right-hand side (an open boundary face copies its interior neighbour)
void L_adjf_box_gather(cudaStream_t st, const Geo& g, int c, const double* faces, double* box);
void L_adjf_box_rhs(cudaStream_t st, const Geo& g, int c, const double* lus, double* box, double* lun);
// pointwise stages: rho_G^{n+1}, the pinned saturation values, the mixture properties, and
// the alpha source with J, the mdot cap and the block sums of the K normalisation
void L_adjf_rhoG(cudaStream_t st, const Geo& g, const Phys& p, const double* T1, const double* w1, const double* lrgn,
                 double* lT1, double* lW1);
void L_adjf_yq(cudaStream_t st, const Geo& g, const Phys& p, const double* T1, const double* alpha1,
               const double* lyq, double* lT1);
void L_adjf_props(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T);
void L_adjf_source(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T,
                   const double* mraw, const double* scal, double jweight, double* mrbar, double* part);

// forward check of the adjoint's stage formulas: max |formula - forward value| and max
// |forward value| per slot (a slot's mom / energy / species / pressure entry is followed
// by its rhs and coupling entries)
enum { CHK_FL = 0, CHK_AF, CHK_AL, CHK_RP, CHK_RM, CHK_ALPHA1, CHK_MRAW, CHK_ENERGY, CHK_ENERGY_R, CHK_ENERGY_C,
       CHK_SPECIES, CHK_SPECIES_R, CHK_SPECIES_C, CHK_MOM, CHK_MOM_R, CHK_MOM_C, CHK_POISSON, CHK_POISSON_R,
       CHK_POISSON_C, CHK_CORRECT, CHK_COUNT };
void L_chk_cells(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const double* mraw,
                 unsigned long long* chk);
void L_chk_faces(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, double* const unew[3],
                 unsigned long long* chk);
void L_chk_rows(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, int kind, const double* D,
                double* const C[3], const double* rhs, unsigned long long* chk);

// ---- linear solvers (solver.cu)
// Box operator on dims m: y_P = D_P x_P + sum_a [c_a[P](x_P - x_{P-e_a}) + c_a[P+e_a](x_P - x_{P+e_a})],
// the coupling of a pair stored at its high cell (c_a[P] = 0 when P_a = 0).
// where the step keeps a solve's statistics (iterations, relative residual, the
// not-converged flag); scal == nullptr: nowhere
struct RecordSpec {
  double* scal;
  int its, res, acc;
};

struct BoxSys {
  int m[3];
  long long N;
  double* D;
  double* c[3];     // c[2] may be null (2D)
  double* b;
  double* x;
};

struct SolveStats {
  int its;
  double relres;
  int converged;
};

struct MGLevel {
  int m[3];
  long long N;
  void* D;          // float or double per precision
  void* c[3];
  void* x;
  void* b;
  void* idg;        // 1 / (D + sum of adjacent couplings), used by the smoother
  void* xp;         // post-smoothed iterate (tiled persistent V-cycle); b by colour (launched)
  int split = 0;    // launched V-cycle, above its tail: idg and the copy of b by colour
};

class Solver {
 public:
  // workspace sized for boxes of up to maxN unknowns
  int setup(long long maxN, cudaStream_t st);
  void release();
  // Jacobi-preconditioned CG; x holds the initial guess and receives the solution
  int pcg_jacobi(const BoxSys& s, double rtol, int maxit, SolveStats* out);
  // multigrid-preconditioned CG on the pressure box (hierarchy built from s)
  int pcg_mg(const BoxSys& s, double rtol, int maxit, int fp32, SolveStats* out);
  // allocate the multigrid hierarchy for a box (outside any stream capture)
  int prepare_mg(const int m[3], int fp32);
  // store the last solve's iterations (slot_its, accumulated when accumulate = 1), relative
  // residual (slot_res, may be null) and a not-converged mark (scal[SC_NC]) on the device
  void record(double* scal, int slot_its, int slot_res, int accumulate);
  // statistics slots of the next solve (set before it; a persistent solve writes them
  // itself and the record() after it then launches nothing)
  void record_next(double* scal, int slot_its, int slot_res, int accumulate) {
    rec_scal = scal; rec_its = slot_its; rec_res = slot_res; rec_acc = accumulate;
  }
  cudaStream_t stream = nullptr;
  cudaStream_t stream2 = nullptr;   // captures the bodies of the device-driven solver loops
  bool capturing = false;           // the step is being captured into a CUDA graph
  bool f32_helm = false;            // Jacobi-PCG as FP32 defect correction (set before setup)
  bool persistent = false;          // MG-PCG in one cooperative launch (set before setup)
  bool persist_pcg = false;         // Jacobi-PCG in one cooperative launch (set before setup)
  int nsys_extra = 0;               // further systems a joint persistent solve may carry (set before setup)
  // K (<= 1 + nsys_extra) independent Helmholtz systems in one persistent launch; the
  // statistics of system k go to recs[k]
  int pcg_jacobi_multi(const BoxSys* s, int K, double rtol, int maxit, const RecordSpec* recs, SolveStats* out);
  long long spin_limit = 1LL << 22;   // polls of a persistent solve's grid-barrier wait before it gives up
  int sm_budget = 0;                // SMs the persistent solves may use (0: the whole GPU)
  int pcg_budget = 0;               // SMs the persistent Jacobi-PCG may use (0: sm_budget)
  int mg_tile[2] = {32, 32};        // tile of the persistent MG's temporal blocking (autotuned)
  size_t pmg_smem_max = 0;          // dynamic shared memory the persistent MG may request
  static constexpr long long PERSIST_MAX_CELLS = 1LL << 22;   // persistent MG: latency-bound sizes only
  // persistent FP32 Jacobi-PCG: one fused pass and one grid barrier per iteration pays at
  // every size (32-bit cell indices); the FP64 one (one block per SM) only up to
  // PERSIST_MAX_CELLS
  static constexpr long long PERSIST_PCG_MAX_CELLS = 1LL << 30;
  int rb = RED_BLOCKS;              // block cap of the reduction kernels (tuned for batches)
  Prof* prof = nullptr;
  // grid of the launched CG kernels (k_pcg_init, k_spmv_dot, k_update and those paired with
  // them, cg_grid): the reduction cap, and at most the CG_BLOCKS_PER_SM blocks per SM their
  // register bound keeps resident, so that the grid-stride loops run as one full wave
  static constexpr int CG_BLOCKS_PER_SM = 6;

 private:
  template <typename F>
  int device_loop(F body);
  int pcg_jacobi_f32(const BoxSys& s, double rtol, int maxit, SolveStats* out);
  template <typename T>
  int pcg_persist(const BoxSys* s, int K, double rtol, int maxit, const RecordSpec* recs, SolveStats* out);
  int persist_blocks(bool f32);
  int cg_grid(long long N);
  RecordSpec take_record();
  double* rec_scal = nullptr;
  int rec_its = 0, rec_res = -1, rec_acc = 0;
  bool recorded = false;
  template <typename T>
  int pcg_mg_persist(const BoxSys& s, double rtol, int maxit, SolveStats* out);
  int pmg_blocks = 0;           // co-resident blocks of the persistent MG-PCG
  int nsm_ = 1;                 // SMs of the device
  double* mg_q2 = nullptr;      // second buffer of its q = A p
  float *fD = nullptr, *fc[3] = {nullptr, nullptr, nullptr}, *fidg = nullptr, *fr = nullptr, *fz = nullptr,
        *fp = nullptr, *fAp = nullptr, *fdx = nullptr;
  static constexpr int PERSIST_VECTORS = 13;
  void* pw[PERSIST_VECTORS] = {};   // persistent-solve vectors
  void* pwx[2][PERSIST_VECTORS] = {};   // those of the second and third system of a joint solve
  unsigned* bar = nullptr;      // grid barrier counter and generation
  int* err = nullptr;           // set when a grid barrier wait ran out
  int pb_f32 = 0, pb_f64 = 0;   // co-resident blocks of the persistent solver
  int build_mg(const BoxSys& s, int fp32);
  void vcycle(int fp32, bool casts);
  long long cap = 0;
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *idg = nullptr;
  double* adg = nullptr;        // total diagonal of the launched FP64 solves' operator (diagonal form)
  double* part = nullptr;       // reduction partials
  double* sc = nullptr;         // device scalars
  int* done = nullptr;
  unsigned* cnt = nullptr;      // last-block ticket counter of the fused reductions
  double* hsc = nullptr;        // pinned host copy of the scalars
  // multigrid
  int nlev = 0;
  MGLevel lev[24];
  void* mgbuf = nullptr;
  size_t mgbytes = 0;
  int mg_fp32 = -1;
  int mg_m[3] = {0, 0, 0};
};

}  // namespace dg
