// api.cu -- problem context, solver orchestration and the C ABI (pint.h).
//
// Flow of one solve (Sec. 3-4 of the paper):
//   FP64 FGMRES(m) on the KKT system of Eq. FinalA (matrix-free matvec)
//     z = P^{-1} v :  r^ = F v (time DFT, Hermitian half)
//                     Stokes: s^_j = (T_j^l)^{-1} r^_j ; x^_j = GMRES(Z_j, P~_j, s^_j, eps)
//                             y^_j = (T_j^r)^{-1} x^_j                    (Algorithm 2)
//                     Oseen:  y^_j = GMRES(G_j, P~_j^(UZ), r^_j, eps)      (Algorithm 3)
//                     z = Re F^{-1} y^
// Every frequency is processed in the same launches; converged frequencies
// drop out through a device-side active mask.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dft_tc.h"
#include "fields.h"
#include "kernels.h"
#include "krylov.h"
#include "pint.h"
#include "tables.h"

using namespace pint;

namespace {
thread_local std::string g_err;

// Wathen's bounds on the spectrum of diag(M)^{-1} M for the bilinear and
// biquadratic elements (Sec. 3.4 cites them for the Chebyshev iteration).
constexpr double Q2_LMIN = 0.25, Q2_LMAX = 1.5625;
constexpr double Q1_LMIN = 0.25, Q1_LMAX = 2.25;

struct Status {
  pint_status code;
  std::string msg;
};
}  // namespace

struct pint_ctx;

// One frequency of a context's frequency-domain solve: the problem it comes
// from (tau, beta, number of time blocks K) and its index j <= K/2.
struct FreqDesc {
  double tau, beta;
  int K, j;
};

template <class T>
struct Engine {
  pint_ctx* c = nullptr;
  Tabs<T> tabs{};
  cpx<T>* R = nullptr;  // frequency vectors [J][nblk]
  cpx<T>* Y = nullptr;
  cpx<T>* T1 = nullptr;
  cpx<T>* T2 = nullptr;
  cpx<T>* T3 = nullptr;
  cpx<T>* V = nullptr;  // inner GMRES basis [m+1][J][nblk]
  cpx<T>* Z = nullptr;  // [m][J][nblk]
  cpx<T>* mgws = nullptr;
  cpx<T>* mgws_q1 = nullptr;  // pressure multigrid workspace when it runs beside the velocity one
  cpx<T>* chebws = nullptr;
  T* cosk = nullptr;
  T* sink = nullptr;

  const T* n2d[PINT_MAXLEV] = {};  // per-level Q2 convection stencils (conv only)
  const T* np2d = nullptr;         // finest-level Q1 convection stencils (conv only)
  int active_freqs = 0;            // frequencies still active in the inner solve (0: all / unknown)
  int active_jobs(int njobs, const int* active) const {
    return active && active_freqs > 0 && active_freqs < c_J() ? std::max(1, (int)((long long)njobs * active_freqs / c_J()))
                                                              : 0;
  }
  int c_J() const;
  // fraction of the frequencies whose work a masked launch does
  double afrac(const int* active) const;
  void mg(int space, bool conv, const FieldJob* jobs, int njobs, cpx<T>* xb, const cpx<T>* bb, const int* active,
          int fields_per_job = 2, cudaStream_t stream = nullptr, cpx<T>* ws = nullptr);
  void cheb(int space, const FieldJob* jobs, int njobs, cpx<T>* xb, const cpx<T>* bb, const int* active,
            int fields_per_job = 2, cudaStream_t stream = nullptr);
  void block_prec(const cpx<T>* U, cpx<T>* Out, const int* active);
  void block_matvec(const BlkCoef* coef, const cpx<T>* X, cpx<T>* Out, const int* active);
  void inner_solve(const cpx<T>* S, cpx<T>* X, int* its_host);
  void freq_solve(cpx<T>* Rin, cpx<T>* Out, int* its_host);
  void apply(const double* r, double* z, int* its_host);
};

struct pint_ctx {
  pint_params p{};
  cudaStream_t st = nullptr;
  int N = 0, K = 0, J = 0, nlev = 0, m_in = 0;
  Slots s{};
  bool oseen = false, conv = false, fp32 = false;
  double omega_conv = 1.0;                // SOR relaxation of the Q_j, Q_j^H multigrids (Oseen)
  // Role in the serving loop's shared frequency solves: 0 = ordinary handle;
  // 1 = member (time-domain parts and the frequency vectors of its DFT only;
  // its frequency solves run in a shared context); 2 = shared frequency-domain
  // context for up to `role_cap` frequencies (no DFT, no outer FGMRES).
  int role = 0, role_cap = 0;
  struct BatchGroup* group = nullptr;     // role 1: the shared context's group
  bool in_solve = false;
  pint_status batch_rc = PINT_OK;         // role 1: status of the last shared frequency solve
  bool gwind = false;                     // conv by node stencils (two-vortex or nodal wind), not separable
  std::vector<double> wind_nodal;         // PINT_WIND_NODAL: [2][n_s] values at the finest Q2 nodes
  double* nst64[PINT_MAXLEV] = {};        // node-order FP64 Q2 convection stencils per level (gwind)
  double* npst64 = nullptr;               // node-order FP64 Q1 convection stencils, finest level (gwind)
  std::vector<void*> allocs;
  size_t dev_bytes = 0;
  std::string err;

  Tabs<double> t64{};
  Tabs<float> t32{};
  MGLayout lay2{}, lay1{};
  long long cheb_per_q2 = 0, cheb_per_q1 = 0;

  OpCoef* d_ops = nullptr;
  int nops = 0;
  double* d_cinv = nullptr;
  BlkCoef* d_blkZ = nullptr;  // inner operator (Z_j Stokes / G_j Oseen)
  BlkCoef* d_blkG = nullptr;  // G_j (Eq. SubBlockG)
  double* d_tc = nullptr;     // Stokes transform constants [J][3]
  double* d_sa = nullptr;     // Stokes Schur combination (1 + c1)   [J] complex
  double* d_sb = nullptr;     // Stokes Schur combination nu c2     [J] complex
  double* d_one = nullptr;    // [J] complex 1
  double* d_invtau = nullptr; // [J] complex 1/tau
  double* d_mtaumu = nullptr; // [J] complex -tau/mu
  double* d_negtau = nullptr; // [J] -tau
  int *d_space = nullptr, *d_conv = nullptr, *d_status = nullptr;  // coarse setup per op
  int jcap = 0;               // frequencies the per-frequency tables and jobs are allocated for
  OpCoef *d_cuza = nullptr, *d_cuzd = nullptr, *d_cmass = nullptr, *d_cxp = nullptr;
  FieldJob *j_W4 = nullptr, *j_Q2 = nullptr, *j_QH2 = nullptr, *j_M2 = nullptr, *j_Kp2 = nullptr,
           *j_Mp2 = nullptr, *j_Kp2s = nullptr, *j_Mp2s = nullptr, *j_one = nullptr;
  int* d_active_one = nullptr;
  GmresState gs{};
  DftTc tc{};              // tensor-core time DFT (FP32 preconditioner), scheme 0 = off
  cudaStream_t st_aux = nullptr;                  // second stream of the Stokes block preconditioner
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int* h_tcerr = nullptr;  // pinned copy of tc.err

  // outer FGMRES (FP64)
  double *oV = nullptr, *oZ = nullptr, *ob = nullptr, *ox = nullptr, *ot = nullptr, *opart = nullptr,
         *oh = nullptr;
  double* ofreq = nullptr;  // FP64 complex [J][nblk] staging for frequency-domain inputs
  double* h_pinned = nullptr;
  int* h_count = nullptr;
  bool have_data = false;

  Engine<double> e64;
  Engine<float> e32;

  // ---- tracing: launch counts per kernel class, event timing for masked classes
  unsigned prof_mask = 0;
  long long prof_launch[PINT_PROF_CLASSES] = {};
  long long prof_syncs = 0;  // host synchronisations of the solve path (pint_profile.host_syncs)
  long long prof_timed[PINT_PROF_CLASSES] = {};
  double prof_ms[PINT_PROF_CLASSES] = {};
  double prof_bytes[PINT_PROF_CLASSES] = {};  // algorithmic bytes (pint.h, pint_profile)
  void add_bytes(int cls, double b) { prof_bytes[cls] += b; }
  struct Pend {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> evpool;
  cudaEvent_t take_event() {
    if (!evpool.empty()) {
      cudaEvent_t e = evpool.back();
      evpool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // Fold completed event pairs into the counters (call after a stream sync).
  void drain() {
    for (auto& q : pend) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) {
        prof_ms[q.cls] += t;
        prof_timed[q.cls]++;
      } else {
        cudaGetLastError();
      }
      evpool.push_back(q.a);
      evpool.push_back(q.b);
    }
    pend.clear();
  }

  // ----------------------------------------------------------- helpers
  pint_status fail(pint_status code, const std::string& m) {
    err = m;
    g_err = m;
    return code;
  }
  bool cu(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    g_err = err;
    return false;
  }
  template <class P>
  bool alloc(P** ptr, size_t bytes) {
    void* v = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&v, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(v);
    dev_bytes += bytes;
    *ptr = static_cast<P*>(v);
    return true;
  }
  template <class P>
  bool upload(P** ptr, const std::vector<P>& host) {
    if (!alloc(ptr, host.size() * sizeof(P))) return false;
    return cudaMemcpy(*ptr, host.data(), host.size() * sizeof(P), cudaMemcpyHostToDevice) == cudaSuccess;
  }
  bool launched(const char* what) { return cu(cudaGetLastError(), what); }
};

template <class T>
int Engine<T>::c_J() const {
  return c->J;
}
template <class T>
double Engine<T>::afrac(const int* active) const {
  return active && active_freqs > 0 ? (double)active_freqs / c->J : 1.0;
}

// algorithmic bytes of operator combinations: every row's operand fields
// read once and its output written once, per (active) frequency
template <class T>
static double combo_bytes(const Engine<T>& e, const ComboArgs<T>& a, const int* active) {
  const double len = a.space == 2 ? (double)e.c->s.ns : (double)e.c->s.nq;
  double f = 0;
  for (int r = 0; r < a.nrows; ++r) f += a.rows[r].nt + a.rows[r].has_z + 1;
  return f * len * 2 * sizeof(T) * e.c->J * e.afrac(active);
}

// RAII scope around the launches of one kernel class: counts nk kernels and,
// if the class is being timed, records a CUDA event pair on the stream.
struct Prof {
  pint_ctx* c;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Prof(pint_ctx* c_, int cls_, int nk, cudaStream_t s_ = nullptr) : c(c_), cls(cls_), s(s_ ? s_ : c_->st) {
    c->prof_launch[cls] += nk;
    if ((c->prof_mask >> cls) & 1u) {
      a = c->take_event();
      cudaEventRecord(a, s);
    }
  }
  ~Prof() {
    if (!a) return;
    cudaEvent_t b = c->take_event();
    cudaEventRecord(b, s);
    c->pend.push_back({cls, a, b});
    if (c->pend.size() > 8192) {
      cudaStreamSynchronize(c->st);
      if (c->st_aux) cudaStreamSynchronize(c->st_aux);
      c->drain();
    }
  }
};
#define PROF_CAT2(a, b) a##b
#define PROF_CAT(a, b) PROF_CAT2(a, b)
#define PROF(ctx, cls, nk) Prof PROF_CAT(prof_scope_, __LINE__)((ctx), (cls), (nk))
#define PROF_ON(ctx, cls, nk, stream) Prof PROF_CAT(prof_scope_, __LINE__)((ctx), (cls), (nk), (stream))

// ============================================================================
// Engine<T>
// ============================================================================
template <class T>
static Tabs<T>& tabs_of(pint_ctx* c);
template <>
Tabs<double>& tabs_of<double>(pint_ctx* c) {
  return c->t64;
}
template <>
Tabs<float>& tabs_of<float>(pint_ctx* c) {
  return c->t32;
}

template <class T>
void Engine<T>::mg(int space, bool conv, const FieldJob* jobs, int njobs, cpx<T>* xb, const cpx<T>* bb,
                   const int* active, int fields_per_job, cudaStream_t stream, cpx<T>* ws) {
  MGLaunch<T> L{};
  L.tabs = tabs;
  L.t64 = c->t64;
  for (int l = 0; l < PINT_MAXLEV; ++l) L.n2d[l] = n2d[l];
  L.fields_per_job = fields_per_job;
  L.cw = c->oseen && space == 2;
  L.lay = space == 2 ? c->lay2 : c->lay1;
  L.ops = c->d_ops;
  L.coarse_inv = c->d_cinv;
  L.jobs = jobs;
  L.njobs = njobs;
  L.xbase = xb;
  L.bbase = bb;
  L.ws = ws ? ws : mgws;
  L.active = active;
  L.cycles = c->p.mg_cycles;
  L.pre = c->p.mg_pre;
  L.post = c->p.mg_post;
  L.omega = c->oseen && space == 2 ? c->omega_conv : c->p.sor_omega;
  L.space = space;
  L.conv = conv;
  L.active_jobs = active_jobs(njobs, active);
  // single-field launches come from the diagnostic component entry points
  // only: fixed CTA size, no tuner entry
  L.no_tune = njobs == 1;
  cudaStream_t st = stream ? stream : c->st;
  {
    const double n = space == 2 ? (double)c->s.ns : (double)c->s.nq;
    c->add_bytes(space == 2 ? PINT_PROF_MG_Q2 : PINT_PROF_MG_Q1,
                 njobs * afrac(active) * (4.0 * (L.pre + L.post) + 8.0) * n * 2 * sizeof(T) * L.cycles);
  }
  PROF_ON(c, space == 2 ? PINT_PROF_MG_Q2 : PINT_PROF_MG_Q1, 1, st);
  launch_mg<T>(L, st);
}

template <class T>
void Engine<T>::cheb(int space, const FieldJob* jobs, int njobs, cpx<T>* xb, const cpx<T>* bb, const int* active,
                     int fields_per_job, cudaStream_t stream) {
  ChebLaunch<T> L{};
  L.tabs = tabs;
  L.t64 = c->t64;
  L.fields_per_job = fields_per_job;
  L.jobs = jobs;
  L.njobs = njobs;
  L.xbase = xb;
  L.bbase = bb;
  L.ws = chebws;
  L.per_job = space == 2 ? c->cheb_per_q2 : c->cheb_per_q1;
  L.active = active;
  L.steps = c->p.cheb_steps;
  L.lmin = space == 2 ? Q2_LMIN : Q1_LMIN;
  L.lmax = space == 2 ? Q2_LMAX : Q1_LMAX;
  L.space = space;
  L.active_jobs = active_jobs(njobs, active);
  c->add_bytes(PINT_PROF_CHEB, njobs * afrac(active) * fields_per_job * 5.0 *
                                   (space == 2 ? (double)c->s.ns : (double)c->s.nq) * 2 * sizeof(T) * L.steps);
  PROF_ON(c, PINT_PROF_CHEB, 1, stream ? stream : c->st);
  launch_cheb<T>(L, stream ? stream : c->st);
}

template <class T>
void Engine<T>::block_matvec(const BlkCoef* coef, const cpx<T>* X, cpx<T>* Out, const int* active) {
  BlkArgs<T> a{};
  a.tabs = tabs;
  a.n2d = n2d[0];
  a.s = c->s;
  a.J = c->J;
  a.nu = c->p.nu;
  a.conv = c->conv;
  a.coef = coef;
  a.active = active;
  a.x = X;
  a.y = Out;
  c->add_bytes(PINT_PROF_BLOCK_MV, c->J * afrac(active) * 2.0 * c->s.nblk * 2 * sizeof(T));
  PROF(c, PINT_PROF_BLOCK_MV, 2);
  launch_block_matvec<T>(a, c->st);
}

// P~_j^{-1} (Stokes, Sec. 3.2) or (P~_j^(UZ))^{-1} (Oseen, Algorithm 3) for
// every frequency: U -> Out.  U and Out must not overlap; T1..T3 are scratch.
template <class T>
void Engine<T>::block_prec(const cpx<T>* U, cpx<T>* Out, const int* active) {
  const int J = c->J;
  const Slots& s = c->s;
  cudaStream_t st = c->st;
  if (!c->oseen) {
    // The velocity and pressure parts of P~_j are independent: the pressure
    // part runs on a second stream beside the velocity multigrid (own
    // workspace; disjoint output slots), joined before returning.
    cudaStream_t sa = c->st_aux;
    cudaEventRecord(c->ev_fork, st);
    cudaStreamWaitEvent(sa, c->ev_fork, 0);
    // W_j^{-1} on the four velocity fields (v and lambda blocks)
    mg(2, false, c->j_W4, 4 * J, Out, U, active, 1);
    // S^_j^{-1} = (1 + c1) K_p^{-1} + nu c2 M_p^{-1} on the p and mu blocks
    mg(1, false, c->j_Kp2, 2 * J, T1, U, active, 1, sa, mgws_q1);
    cheb(1, c->j_Mp2, J, T2, U, active, 2, sa);
    c->add_bytes(PINT_PROF_COMBO, 2 * 3.0 * s.nq * 2 * sizeof(T) * J * afrac(active));
    { PROF_ON(c, PINT_PROF_COMBO, 1, sa); launch_lincomb<T>(J, s.nblk, s.nq, Out, s.p, T1, s.p, c->d_sa, T2, s.p, c->d_sb, active, sa); }
    { PROF_ON(c, PINT_PROF_COMBO, 1, sa); launch_lincomb<T>(J, s.nblk, s.nq, Out, s.mu, T1, s.mu, c->d_sa, T2, s.mu, c->d_sb, active, sa); }
    cudaEventRecord(c->ev_join, sa);
    cudaStreamWaitEvent(st, c->ev_join, 0);
    return;
  }
  // ---- Oseen: Uzawa (Eq. Uzawa11) on G^(1,1), x^(0) = 0
  cudaMemsetAsync(Out, 0, sizeof(cpx<T>) * (size_t)J * s.nblk, st);
  const long long lenv = 2LL * s.ns;
  ComboArgs<T> ca{};
  ca.tabs = tabs;
  ca.n2d = n2d[0];
  ca.np2d = np2d;
  ca.s = s;
  ca.J = J;
  ca.active = active;
  ca.conv = c->conv;
  ca.space = 2;
  for (int step = 0; step < c->p.uzawa_steps; ++step) {
    // T1[v] = b1 - tau M x1 - (d M + tau L)^H x2
    ca.nrows = 2;
    ca.ncoef = 3;
    ca.coef = c->d_cuza;
    ca.rows[0] = ComboRow{s.vx, s.vx, {s.vx, s.lx}, 0, {1, 2}, 2, 1};
    ca.rows[1] = ComboRow{s.vy, s.vy, {s.vy, s.ly}, 0, {1, 2}, 2, 1};
    ca.x = Out;
    ca.z = U;
    ca.out = T1;
    c->add_bytes(PINT_PROF_COMBO, combo_bytes(*this, ca, active));
    { PROF(c, PINT_PROF_COMBO, 1); launch_combo<T>(ca, st); }
    // x1 += (1/tau) M^-1 T1[v]   (M^ = Chebyshev)
    cheb(2, c->j_M2, J, T2, T1, active);
    c->add_bytes(PINT_PROF_COMBO, 3.0 * lenv * 2 * sizeof(T) * J * afrac(active));
    { PROF(c, PINT_PROF_COMBO, 1); launch_lincomb<T>(J, s.nblk, lenv, Out, s.vx, Out, s.vx, c->d_one, T2, s.vx, c->d_invtau, active, st); }
    // T1[lam] = b2 - (d M + tau L) x1 + tau/beta M x2
    ca.coef = c->d_cuzd;
    ca.rows[0] = ComboRow{s.lx, s.lx, {s.vx, s.lx}, 0, {1, 2}, 2, 1};
    ca.rows[1] = ComboRow{s.ly, s.ly, {s.vy, s.ly}, 0, {1, 2}, 2, 1};
    ca.x = Out;
    ca.z = U;
    ca.out = T1;
    c->add_bytes(PINT_PROF_COMBO, combo_bytes(*this, ca, active));
    { PROF(c, PINT_PROF_COMBO, 1); launch_combo<T>(ca, st); }
    // S^^{-1} = tau Q^{-H} M Q^{-1}
    mg(2, c->conv, c->j_Q2, 2 * J, T2, T1, active, 1);
    ca.coef = c->d_cmass;
    ca.ncoef = 2;
    ca.rows[0] = ComboRow{s.lx, 0, {s.lx, 0}, 0, {1, 0}, 1, 0};
    ca.rows[1] = ComboRow{s.ly, 0, {s.ly, 0}, 0, {1, 0}, 1, 0};
    ca.x = T2;
    ca.z = nullptr;
    ca.out = T3;
    c->add_bytes(PINT_PROF_COMBO, combo_bytes(*this, ca, active));
    { PROF(c, PINT_PROF_COMBO, 1); launch_combo<T>(ca, st); }
    mg(2, c->conv, c->j_QH2, 2 * J, T1, T3, active, 1);
    // x2 -= (1/mu) tau Q^{-H} M Q^{-1} (...)
    c->add_bytes(PINT_PROF_COMBO, 3.0 * lenv * 2 * sizeof(T) * J * afrac(active));
    { PROF(c, PINT_PROF_COMBO, 1); launch_lincomb<T>(J, s.nblk, lenv, Out, s.lx, Out, s.lx, c->d_one, T1, s.lx, c->d_mtaumu, active, st); }
  }
  // ---- Algorithm 3: y34 = -S^_j^{-1} (r34 - tau (B y2; B y1))
  BResArgs<T> br{};
  br.tabs = tabs;
  br.s = s;
  br.J = J;
  br.c = -c->p.tau;
  br.cj = c->d_negtau;  // -tau of each frequency's problem
  br.out0 = s.p;
  br.z0 = s.p;
  br.vel0 = s.lx;
  br.out1 = s.mu;
  br.z1 = s.mu;
  br.vel1 = s.vx;
  br.active = active;
  br.x = Out;
  br.z = U;
  br.out = T1;
  c->add_bytes(PINT_PROF_COMBO, 2.0 * (2.0 * s.ns + 2.0 * s.nq) * 2 * sizeof(T) * J * afrac(active));
  {
    PROF(c, PINT_PROF_COMBO, 1);
    launch_bres<T>(br, st);
  }
  // swap + (tau M_p)^{-1}: T2[p] = Cheb(T1[mu]), T2[mu] = Cheb(T1[p]) (1/tau folded below)
  cheb(1, c->j_Mp2s, J, T2, T1, active);
  // X_p, the second swap's sign and the 1/tau factors
  ComboArgs<T> cq{};
  cq.tabs = tabs;
  cq.n2d = n2d[0];
  cq.np2d = np2d;
  cq.s = s;
  cq.J = J;
  cq.active = active;
  cq.conv = c->conv;
  cq.space = 1;
  cq.nrows = 2;
  cq.ncoef = 5;
  cq.coef = c->d_cxp;
  cq.rows[0] = ComboRow{s.p, 0, {s.p, s.mu}, 0, {1, 2}, 2, 0};
  cq.rows[1] = ComboRow{s.mu, 0, {s.p, s.mu}, 0, {3, 4}, 2, 0};
  cq.x = T2;
  cq.z = nullptr;
  cq.out = T3;
  c->add_bytes(PINT_PROF_COMBO, combo_bytes(*this, cq, active));
  { PROF(c, PINT_PROF_COMBO, 1); launch_combo<T>(cq, st); }
  // swap + (tau K_p)^{-1}: Out[p] = MG(T3[mu]), Out[mu] = MG(T3[p])
  mg(1, false, c->j_Kp2s, 2 * J, Out, T3, active, 1);
}

// Inner solve on all frequencies: GMRES(A_j, P_j, S_j, eps) or, for the
// linear variant (Algorithm 1), one application of the block preconditioner.
template <class T>
void Engine<T>::inner_solve(const cpx<T>* S, cpx<T>* X, int* its_host) {
  const int J = c->J;
  const long long nb = c->s.nblk;
  cudaStream_t st = c->st;
  if (c->p.linear) {
    block_prec(S, X, nullptr);
    if (its_host)
      for (int j = 0; j < J; ++j) its_host[j] = 0;
    return;
  }
  GmresState& G = c->gs;
  const int m = G.m;
  const long long hs = (long long)(m + 1) * m * 2;  // H stride per frequency (doubles)
  const size_t vs = (size_t)J * nb;                 // one basis vector (all frequencies)
  const double vbytes = (double)nb * 2 * sizeof(T);  // one frequency's vector
  double its_sum = 0;                                // sum over frequencies of the steps taken
  c->add_bytes(PINT_PROF_INNER, 3.0 * J * vbytes);
  {
    PROF(c, PINT_PROF_INNER, 4);
    launch_bdot<T>(J, nb, S, S, nb, nb, G.partial, G.g, (long long)(m + 1) * 2, nullptr, false, st);
    launch_gmres_start(G, st);
    launch_bscale_inv<T>(J, nb, S, V, nb, G.beta0, 1, G.active, st);
  }
  active_freqs = 0;
  for (int i = 0; i < m; ++i) {
    cpx<T>* Vi = V + (size_t)i * vs;
    cpx<T>* Zi = Z + (size_t)i * vs;
    cpx<T>* Vn = V + (size_t)(i + 1) * vs;
    if (i > 0) active_freqs = *c->h_count;  // still-active frequencies after the previous step
    block_prec(Vi, Zi, G.active);
    block_matvec(c->d_blkZ, Zi, Vn, G.active);
    // classical Gram-Schmidt with one reorthogonalisation (CGS2) against
    // V_0..V_i for all active frequencies, then the norm of the result
    const int cnt = i + 1;
    const double act = J * afrac(G.active);
    its_sum += act;
    c->add_bytes(PINT_PROF_INNER, (4.0 * cnt + 8.0) * act * vbytes);
    const int nk = 2 * ((cnt + 7) / 8 + 1) + 2 * 1 + 1 + 1 + 1 + 1;
    PROF(c, PINT_PROF_INNER, nk + 1);
    launch_bmdot<T>(J, nb, V, (long long)vs, cnt, Vn, G.cpart, G.H, hs, m, i, false, G.active, st);
    launch_hcol_gather(J, cnt, G.H, hs, m, i, G.hc, G.active, st);
    launch_bmaxpy<T>(J, nb, V, (long long)vs, cnt, Vn, G.hc, 256, nullptr, nullptr, 0, G.active, st);
    launch_bmdot<T>(J, nb, V, (long long)vs, cnt, Vn, G.cpart, G.hc2, 256, 1, 0, false, G.active, st);
    double* hn = G.H + ((size_t)(i + 1) * m + i) * 2;
    launch_bmaxpy<T>(J, nb, V, (long long)vs, cnt, Vn, G.hc2, 256, G.npart, hn, hs, G.active, st);
    launch_hcol_add(J, cnt, G.H, hs, m, i, G.hc2, G.active, st);
    launch_bscale_inv<T>(J, nb, Vn, Vn, nb, hn, hs, G.active, st);
    launch_gmres_givens(G, i, c->p.inner_tol, c->p.fixed_inner_its, st);
    cudaMemcpyAsync(c->h_count, G.count, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    ++c->prof_syncs;
    c->drain();
    if (*c->h_count == 0) break;
  }
  active_freqs = 0;
  c->add_bytes(PINT_PROF_INNER, (its_sum + J) * vbytes);
  {
    PROF(c, PINT_PROF_INNER, 2);
    launch_gmres_finish<T>(G, nb, Z, (long long)vs, X, st);
  }
  if (its_host) {
    cudaMemcpyAsync(its_host, G.its, sizeof(int) * J, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
  }
}

template <class T>
void Engine<T>::freq_solve(cpx<T>* Rin, cpx<T>* Out, int* its_host) {
  if (!c->oseen) {
    c->add_bytes(PINT_PROF_COMBO, 2 * 2.0 * c->J * c->s.nblk * 2 * sizeof(T));
    {
      PROF(c, PINT_PROF_COMBO, 1);
      launch_stokes_transform<T>(0, c->J, c->s, c->d_tc, Rin, c->st);
    }
    inner_solve(Rin, Out, its_host);
    {
      PROF(c, PINT_PROF_COMBO, 1);
      launch_stokes_transform<T>(1, c->J, c->s, c->d_tc, Out, c->st);
    }
  } else {
    inner_solve(Rin, Out, its_host);
  }
}

// Time DFT of a [K][nblk] FP64 vector into the Hermitian half [J][nblk] and
// back (Sec. 3.1): tensor cores for the FP32 preconditioner when enabled,
// else the CUDA-core kernels.
// algorithmic bytes of one time DFT: the FP64 time slices once, the
// Hermitian half of the spectrum once in the preconditioner's precision
template <class T>
double dft_bytes(const pint_ctx* c) {
  return 8.0 * c->K * c->s.nblk + (double)c->J * c->s.nblk * 2 * sizeof(T);
}
template <class T>
void dft_forward_any(pint_ctx* c, Engine<T>& e, const double* x, cpx<T>* X) {
  c->add_bytes(PINT_PROF_DFT_FWD, dft_bytes<T>(c));
  PROF(c, PINT_PROF_DFT_FWD, 1);
  launch_dft_forward<T>(c->K, c->J, c->s.nblk, x, X, e.cosk, e.sink, c->st);
}
template <>
void dft_forward_any<float>(pint_ctx* c, Engine<float>& e, const double* x, cpx<float>* X) {
  c->add_bytes(PINT_PROF_DFT_FWD, dft_bytes<float>(c));
  PROF(c, PINT_PROF_DFT_FWD, 1);
  if (c->tc.scheme)
    launch_dft_tc_forward(c->tc, c->s.nblk, x, X, c->st);
  else
    launch_dft_forward<float>(c->K, c->J, c->s.nblk, x, X, e.cosk, e.sink, c->st);
}
template <class T>
void dft_inverse_any(pint_ctx* c, Engine<T>& e, const cpx<T>* X, double* y) {
  c->add_bytes(PINT_PROF_DFT_INV, dft_bytes<T>(c));
  PROF(c, PINT_PROF_DFT_INV, 1);
  launch_dft_inverse<T>(c->K, c->J, c->s.nblk, X, y, e.cosk, e.sink, c->st);
}
template <>
void dft_inverse_any<float>(pint_ctx* c, Engine<float>& e, const cpx<float>* X, double* y) {
  c->add_bytes(PINT_PROF_DFT_INV, dft_bytes<float>(c));
  PROF(c, PINT_PROF_DFT_INV, 1);
  if (c->tc.scheme)
    launch_dft_tc_inverse(c->tc, c->s.nblk, X, y, c->st);
  else
    launch_dft_inverse<float>(c->K, c->J, c->s.nblk, X, y, e.cosk, e.sink, c->st);
}

// The frequency solves of a member of the serving loop's shared solves
// (role 1), run together with those of the other members in a shared
// context; defined with the serving support below.
pint_status shared_freq_solve(pint_ctx* c, void* R, void* Y, int* its_host);

template <class T>
void Engine<T>::apply(const double* r, double* z, int* its_host) {
  dft_forward_any<T>(c, *this, r, R);
  if (c->role == 1)
    c->batch_rc = shared_freq_solve(c, R, Y, its_host);
  else
    freq_solve(R, Y, its_host);
  dft_inverse_any<T>(c, *this, Y, z);
}

// ============================================================================
// setup
// ============================================================================
namespace {

bool valid_params(const pint_params* p, std::string& why) {
  if (!p) return why = "null params", false;
  if (p->kind != PINT_STOKES && p->kind != PINT_OSEEN) return why = "kind must be PINT_STOKES or PINT_OSEEN", false;
  if (p->level < 1 || p->level > 10) return why = "level must be in [1, 10]", false;
  if (!(p->x1 > p->x0)) return why = "x1 must exceed x0", false;
  if (p->n_t < 1 || p->n_t > 4096) return why = "n_t must be in [1, 4096]", false;
  if (!(p->tau > 0) || !(p->beta > 0) || !(p->nu > 0)) return why = "tau, beta, nu must be positive", false;
  if (p->wind != PINT_WIND_NONE && p->wind != PINT_WIND_RECIRC && p->wind != PINT_WIND_TWO_VORTEX &&
      p->wind != PINT_WIND_NODAL)
    return why = "unknown wind", false;
  if ((p->wind == PINT_WIND_RECIRC || p->wind == PINT_WIND_TWO_VORTEX) && (p->x0 != -1.0 || p->x1 != 1.0))
    return why = "the built-in winds are defined on the domain [-1,1]^2", false;
  if (p->prec != PINT_PREC_FP64 && p->prec != PINT_PREC_FP32) return why = "unknown precision", false;
  if (p->dft_mode < PINT_DFT_AUTO || p->dft_mode > PINT_DFT_TF32X3) return why = "unknown dft_mode", false;
  if ((p->dft_mode == PINT_DFT_BF16X6 || p->dft_mode == PINT_DFT_TF32X3) &&
      (p->prec != PINT_PREC_FP32 || p->n_t > 256))
    return why = "tensor-core DFT modes need prec = PINT_PREC_FP32 and n_t <= 256", false;
  if (p->outer_restart < 1 || p->outer_restart > 200) return why = "outer_restart must be in [1, 200]", false;
  if (p->outer_maxit < 1) return why = "outer_maxit must be positive", false;
  if (!(p->outer_tol > 0)) return why = "outer_tol must be positive", false;
  if (p->inner_maxit < 1 || p->inner_maxit > 127) return why = "inner_maxit must be in [1, 127]", false;
  if (p->fixed_inner_its < 0 || p->fixed_inner_its > 127) return why = "fixed_inner_its must be in [0, 127]", false;
  if (!(p->inner_tol >= 0)) return why = "inner_tol must be >= 0", false;
  if (p->mg_cycles < 1 || p->mg_pre < 0 || p->mg_post < 0 || p->cheb_steps < 1 || p->uzawa_steps < 1)
    return why = "multigrid / Chebyshev / Uzawa counts must be positive", false;
  if (!(p->uzawa_mu > 0) || !(p->sor_omega > 0) || !(p->sor_omega < 2))
    return why = "uzawa_mu must be positive and sor_omega in (0, 2)", false;
  if (!(p->sor_omega_conv >= 0) || !(p->sor_omega_conv < 2))
    return why = "sor_omega_conv must be 0 (same as sor_omega) or in (0, 2)", false;
  return true;
}

inline std::vector<double> cplx_table(int J, double re, double im) {
  std::vector<double> v(2 * (size_t)J);
  for (int j = 0; j < J; ++j) {
    v[2 * j] = re;
    v[2 * j + 1] = im;
  }
  return v;
}

template <class T>
bool setup_engine(pint_ctx* c, Engine<T>& e, size_t mg_jobs_q2, size_t mg_jobs_q1, size_t cheb_jobs_q2,
                  size_t cheb_jobs_q1) {
  e.c = c;
  e.tabs = tabs_of<T>(c);
  const size_t fv = (size_t)c->J * c->s.nblk;
  if (!c->alloc(&e.R, fv * sizeof(cpx<T>)) || !c->alloc(&e.Y, fv * sizeof(cpx<T>))) return false;
  if (c->role == 1) {
    // a member of the shared frequency solves: the DFT's input and output only
    std::vector<T> cs(c->K), sn(c->K);
    for (int k = 0; k < c->K; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)c->K;
      cs[k] = (T)std::cos(a);
      sn[k] = (T)std::sin(a);
    }
    return c->upload(&e.cosk, cs) && c->upload(&e.sink, sn);
  }
  if (!c->alloc(&e.T1, fv * sizeof(cpx<T>)) || !c->alloc(&e.T2, fv * sizeof(cpx<T>)) ||
      !c->alloc(&e.T3, fv * sizeof(cpx<T>)))
    return false;
  if (!c->p.linear) {
    const int m = c->m_in;
    if (!c->alloc(&e.V, (size_t)(m + 1) * fv * sizeof(cpx<T>)) || !c->alloc(&e.Z, (size_t)m * fv * sizeof(cpx<T>)))
      return false;
  }
  const size_t mgws = std::max(mg_jobs_q2 * (size_t)c->lay2.per_job, mg_jobs_q1 * (size_t)c->lay1.per_job);
  const size_t chws = std::max(cheb_jobs_q2 * (size_t)c->cheb_per_q2, cheb_jobs_q1 * (size_t)c->cheb_per_q1);
  if (!c->alloc(&e.mgws, mgws * sizeof(cpx<T>)) || !c->alloc(&e.chebws, chws * sizeof(cpx<T>))) return false;
  if (!c->oseen && !c->alloc(&e.mgws_q1, mg_jobs_q1 * (size_t)c->lay1.per_job * sizeof(cpx<T>))) return false;
  if (c->conv) {
    T* t = nullptr;
    if (!c->alloc(&t, (size_t)c->s.nq * 9 * sizeof(T))) return false;
    launch_build_np2d<T>(c->t64, t, c->gwind ? c->npst64 : nullptr, c->st);
    e.np2d = t;
  }
  if (c->conv)
    for (int l = 0; l < c->nlev; ++l) {
      const size_t n2 = 2 * (size_t)(c->N >> l) + 1, w6 = (n2 + 5) / 6;
      T* t = nullptr;
      if (!c->alloc(&t, 36 * w6 * w6 * 25 * sizeof(T))) return false;
      launch_build_n2d<T>(c->t64, l, t, c->gwind ? c->nst64[l] : nullptr, c->st);
      e.n2d[l] = t;
    }
  std::vector<T> cs(c->K), sn(c->K);
  for (int k = 0; k < c->K; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)c->K;
    cs[k] = (T)std::cos(a);
    sn[k] = (T)std::sin(a);
  }
  return c->upload(&e.cosk, cs) && c->upload(&e.sink, sn);
}

MGLayout make_layout(int nlev, int N, int space) {
  MGLayout L{};
  L.nlev = nlev;
  long long off = 0;
  for (int l = 0; l < nlev; ++l) {
    const int Nl = N >> l;
    L.n[l] = space == 2 ? 2 * Nl + 1 : Nl + 1;
  }
  // Q2 fields run in the class-blocked layout (36 classes of ceil(n/6)^2
  // nodes), so level 0 is copied too
  auto lsize = [&](int l) -> long long {
    if (space == 2) {
      // class-blocked layout, or the padded per-type layout of the
      // compile-time-sized kernel, whichever is larger
      const long long w6 = (L.n[l] + 5) / 6, Nl = N >> l;
      return std::max(36 * w6 * w6, 4 * (Nl + 1) * (long long)q2p_pitch((int)Nl));
    }
    return (long long)L.n[l] * L.n[l];
  };
  for (int l = space == 2 ? 0 : 1; l < nlev; ++l) {
    const long long sz = lsize(l);
    L.off_x[l] = off;
    off += sz;
    L.off_b[l] = off;
    off += sz;
  }
  for (int l = 0; l + 1 < nlev; ++l) {
    L.off_r[l] = off;
    off += lsize(l);
  }
  L.per_job = off > 0 ? off : 1;
  return L;
}

// Convection stencils of the two-vortex or nodal wind on level l of p's grid
// hierarchy (the nodal wind injected from the finest grid).
void level_convection_stencils(const pint_params& p, const double* wind, int l, std::vector<double>& q2,
                               std::vector<double>& q1) {
  const int N = 1 << p.level;
  if (p.wind == PINT_WIND_NODAL) {
    const int nf = 2 * N + 1, nl = 2 * (N >> l) + 1, r = 1 << l;
    std::vector<double> wl(2 * (size_t)nl * nl);
    for (int comp = 0; comp < 2; ++comp)
      for (int iy = 0; iy < nl; ++iy)
        for (int ix = 0; ix < nl; ++ix)
          wl[((size_t)comp * nl + iy) * nl + ix] = wind[((size_t)comp * nf + (size_t)iy * r) * nf + (size_t)ix * r];
    build_nodal_wind_stencils(N >> l, p.x0, p.x1, wl.data(), q2, q1);
  } else {
    build_two_vortex_stencils(N >> l, p.x0, p.x1, q2, q1);
  }
}

// ---------------------------------------------------------------------------
// Per-frequency tables.  A context's frequency-domain solve runs over a list
// of frequencies, each from a problem with its own tau, beta and number of
// time blocks K (one problem for a handle; several for the shared solve of
// the serving loop, whose members share grid, wind, nu and solver settings).
// The tables are allocated for `cap` frequencies once and refilled.
// ---------------------------------------------------------------------------
bool alloc_freq_tables(pint_ctx* c, int cap) {
  const size_t nops = 2 * (size_t)cap + 3;
  bool ok = c->alloc(&c->d_ops, sizeof(OpCoef) * nops) && c->alloc(&c->d_space, sizeof(int) * nops) &&
            c->alloc(&c->d_conv, sizeof(int) * nops) && c->alloc(&c->d_status, sizeof(int) * nops) &&
            c->alloc(&c->d_cinv, sizeof(double) * 2 * PINT_NC_MAX * PINT_NC_MAX * nops) &&
            c->alloc(&c->d_blkZ, sizeof(BlkCoef) * cap) && c->alloc(&c->d_blkG, sizeof(BlkCoef) * cap) &&
            c->alloc(&c->d_tc, sizeof(double) * 3 * cap) && c->alloc(&c->d_sa, sizeof(double) * 2 * cap) &&
            c->alloc(&c->d_sb, sizeof(double) * 2 * cap) && c->alloc(&c->d_one, sizeof(double) * 2 * cap) &&
            c->alloc(&c->d_invtau, sizeof(double) * 2 * cap) && c->alloc(&c->d_mtaumu, sizeof(double) * 2 * cap) &&
            c->alloc(&c->d_negtau, sizeof(double) * cap) && c->alloc(&c->d_cuza, sizeof(OpCoef) * 3 * cap) &&
            c->alloc(&c->d_cuzd, sizeof(OpCoef) * 3 * cap) && c->alloc(&c->d_cmass, sizeof(OpCoef) * 2 * cap) &&
            c->alloc(&c->d_cxp, sizeof(OpCoef) * 5 * cap);
  const size_t fj = sizeof(FieldJob);
  if (!c->oseen)
    ok = ok && c->alloc(&c->j_W4, fj * 4 * cap) && c->alloc(&c->j_Kp2, fj * 2 * cap) &&
         c->alloc(&c->j_Mp2, fj * cap);
  else
    ok = ok && c->alloc(&c->j_Q2, fj * 2 * cap) && c->alloc(&c->j_QH2, fj * 2 * cap) &&
         c->alloc(&c->j_M2, fj * cap) && c->alloc(&c->j_Kp2s, fj * 2 * cap) && c->alloc(&c->j_Mp2s, fj * cap);
  ok = ok && c->alloc(&c->j_one, fj) && c->alloc(&c->d_active_one, sizeof(int) * cap);
  c->jcap = cap;
  return ok;
}

template <class V>
bool put(pint_ctx* c, V* dst, const std::vector<V>& src) {
  return c->cu(cudaMemcpyAsync(dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice, c->st), "tables");
}

pint_status fill_freq_tables(pint_ctx* c, const std::vector<FreqDesc>& fd) {
  const int J = (int)fd.size();
  if (J < 1 || J > c->jcap) return c->fail(PINT_ERR_ARG, "frequency list exceeds the context's capacity");
  c->J = J;
  c->gs.J = J;
  const pint_params& p = c->p;
  const Slots& s = c->s;
  const double nu = p.nu, mu = p.uzawa_mu;
  std::vector<double> dr(J), dc(J), c1(J), c2(J);
  for (int j = 0; j < J; ++j) {
    const double tau = fd[j].tau, beta = fd[j].beta;
    const double th = 2.0 * M_PI * (double)fd[j].j / (double)fd[j].K;
    dr[j] = 1.0 - std::cos(th);  // d_j = 1 - exp(-2 pi i j / K)
    dc[j] = std::sin(th);
    c1[j] = dr[j] / std::sqrt(tau * tau / beta + dc[j] * dc[j]);
    c2[j] = 1.0 / std::sqrt(1.0 / beta + dc[j] * dc[j] / (tau * tau));
  }
  // operators: [0, J): W_j (Stokes) / Q_j (Oseen); [J, 2J): Q_j^H; 2J: K_p; 2J+1: M; 2J+2: M_p
  c->nops = 2 * J + 3;
  std::vector<OpCoef> ops(c->nops, OpCoef{0, 0, 0, 0});
  std::vector<int> space(c->nops, 0), convf(c->nops, 0);
  for (int j = 0; j < J; ++j) {
    const double tau = fd[j].tau, sb = 1.0 / std::sqrt(fd[j].beta);
    if (!c->oseen) {
      ops[j] = OpCoef{1.0 + c1[j], 0.0, c2[j] * nu, 0.0};  // W_j = (1 + c1) M + c2 nu K
      space[j] = 2;
    } else {
      // Q_j = d_j M + tau (nu K + N) + tau/sqrt(beta) M ; Q_j^H with N^T = -N
      ops[j] = OpCoef{dr[j] + tau * sb, dc[j], tau * nu, tau};
      ops[J + j] = OpCoef{dr[j] + tau * sb, -dc[j], tau * nu, -tau};
      space[j] = space[J + j] = 2;
      convf[j] = convf[J + j] = c->conv ? 1 : 0;
    }
  }
  ops[2 * J] = OpCoef{0.0, 0.0, 1.0, 0.0};
  space[2 * J] = 1;
  ops[2 * J + 1] = OpCoef{1.0, 0.0, 0.0, 0.0};
  ops[2 * J + 2] = OpCoef{1.0, 0.0, 0.0, 0.0};
  if (!put(c, c->d_ops, ops) || !put(c, c->d_space, space) || !put(c, c->d_conv, convf) ||
      !c->cu(cudaMemsetAsync(c->d_status, 0, sizeof(int) * c->nops, c->st), "coarse status"))
    return PINT_ERR_CUDA;
  launch_coarse_setup(c->t64, c->d_ops, c->d_space, c->d_conv, c->nops, c->d_cinv, c->d_status,
                      c->gwind ? c->nst64[c->nlev - 1] : nullptr, c->st);
  if (!c->launched("coarse setup")) return PINT_ERR_CUDA;

  // frequency-block coefficients: G_j (Eq. SubBlockG) and Z_j (Eq. GJTransformation)
  std::vector<BlkCoef> bz(J), bg(J);
  std::vector<double> tc(3 * (size_t)J), sa(2 * (size_t)J), sbv(2 * (size_t)J), one(2 * (size_t)J),
      invtau(2 * (size_t)J), mtaumu(2 * (size_t)J), negtau(J);
  std::vector<OpCoef> cuza(3 * (size_t)J), cuzd(3 * (size_t)J), cmass(2 * (size_t)J), cxp(5 * (size_t)J);
  for (int j = 0; j < J; ++j) {
    const double tau = fd[j].tau, beta = fd[j].beta;
    // a12 = conj(d_j), a21 = d_j with d_j = dr + i dc
    bg[j] = BlkCoef{tau, 0, dr[j], -dc[j], dr[j], dc[j], -tau / beta, 0, tau, tau, tau, 0};
    bz[j] = c->oseen ? bg[j] : BlkCoef{1, 0, c1[j], 0, c1[j], 0, -1, 0, c2[j], c2[j], 1, 0};
    tc[3 * j] = std::sqrt(tau);
    tc[3 * j + 1] = dc[j];
    tc[3 * j + 2] = c2[j];
    sa[2 * j] = 1.0 + c1[j];
    sa[2 * j + 1] = 0;
    sbv[2 * j] = nu * c2[j];
    sbv[2 * j + 1] = 0;
    one[2 * j] = 1.0;
    one[2 * j + 1] = 0.0;
    invtau[2 * j] = 1.0 / tau;
    invtau[2 * j + 1] = 0.0;
    mtaumu[2 * j] = -tau / mu;
    mtaumu[2 * j + 1] = 0.0;
    negtau[j] = -tau;
    // Oseen combination coefficients
    // T1[v] = 1 b1 + (-tau M) x1 + (-(conj d) M - tau nu K + tau N) x2
    cuza[3 * j + 0] = OpCoef{1, 0, 0, 0};
    cuza[3 * j + 1] = OpCoef{-tau, 0, 0, 0};
    cuza[3 * j + 2] = OpCoef{-dr[j], dc[j], -tau * nu, tau};
    // T1[lam] = 1 b2 + (-d M - tau nu K - tau N) x1 + (tau/beta M) x2
    cuzd[3 * j + 0] = OpCoef{1, 0, 0, 0};
    cuzd[3 * j + 1] = OpCoef{-dr[j], -dc[j], -tau * nu, -tau};
    cuzd[3 * j + 2] = OpCoef{tau / beta, 0, 0, 0};
    cmass[2 * j + 0] = OpCoef{0, 0, 0, 0};
    cmass[2 * j + 1] = OpCoef{1, 0, 0, 0};
    // T3[p] = -(1/tau^2) [tau M_p a + (conj(d) M_p + tau nu K_p - tau N_p) b]
    // T3[mu] = -(1/tau^2) [(d M_p + tau nu K_p + tau N_p) a - tau/beta M_p b]
    const double it2 = 1.0 / (tau * tau);
    cxp[5 * j + 0] = OpCoef{0, 0, 0, 0};
    cxp[5 * j + 1] = OpCoef{-1.0 / tau, 0, 0, 0};
    cxp[5 * j + 2] = OpCoef{-dr[j] * it2, dc[j] * it2, -nu / tau, 1.0 / tau};
    cxp[5 * j + 3] = OpCoef{-dr[j] * it2, -dc[j] * it2, -nu / tau, -1.0 / tau};
    cxp[5 * j + 4] = OpCoef{1.0 / (beta * tau), 0, 0, 0};
  }
  if (!put(c, c->d_blkZ, bz) || !put(c, c->d_blkG, bg) || !put(c, c->d_tc, tc) || !put(c, c->d_sa, sa) ||
      !put(c, c->d_sb, sbv) || !put(c, c->d_one, one) || !put(c, c->d_invtau, invtau) ||
      !put(c, c->d_mtaumu, mtaumu) || !put(c, c->d_negtau, negtau) || !put(c, c->d_cuza, cuza) ||
      !put(c, c->d_cuzd, cuzd) || !put(c, c->d_cmass, cmass) || !put(c, c->d_cxp, cxp))
    return PINT_ERR_CUDA;

  // ---- job tables: each job the (x slot, b slot) pairs of one frequency sharing one operator
  using SlotPairs = std::vector<std::pair<long long, long long>>;
  auto jobs = [&](std::vector<SlotPairs> groups, int opbase, bool per_j_op) {
    std::vector<FieldJob> v;
    for (int j = 0; j < J; ++j)
      for (auto& grp : groups) {
        FieldJob jb{};
        jb.nf = (int)grp.size();
        for (int f = 0; f < jb.nf; ++f) {
          jb.x_off[f] = (long long)j * s.nblk + grp[f].first;
          jb.b_off[f] = (long long)j * s.nblk + grp[f].second;
        }
        jb.op = per_j_op ? opbase + j : opbase;
        jb.freq = j;
        v.push_back(jb);
      }
    return v;
  };
  bool ok = true;
  if (!c->oseen) {
    ok = put(c, c->j_W4, jobs({{{s.vx, s.vx}}, {{s.vy, s.vy}}, {{s.lx, s.lx}}, {{s.ly, s.ly}}}, 0, true)) &&
         put(c, c->j_Kp2, jobs({{{s.p, s.p}}, {{s.mu, s.mu}}}, 2 * J, false)) &&
         put(c, c->j_Mp2, jobs({{{s.p, s.p}, {s.mu, s.mu}}}, 2 * J + 2, false));
  } else {
    ok = put(c, c->j_Q2, jobs({{{s.lx, s.lx}}, {{s.ly, s.ly}}}, 0, true)) &&
         put(c, c->j_QH2, jobs({{{s.lx, s.lx}}, {{s.ly, s.ly}}}, J, true)) &&
         put(c, c->j_M2, jobs({{{s.vx, s.vx}, {s.vy, s.vy}}}, 2 * J + 1, false)) &&
         put(c, c->j_Kp2s, jobs({{{s.p, s.mu}}, {{s.mu, s.p}}}, 2 * J, false)) &&
         put(c, c->j_Mp2s, jobs({{{s.p, s.mu}, {s.mu, s.p}}}, 2 * J + 2, false));
  }
  if (!ok) return PINT_ERR_CUDA;
  {
    std::vector<int> st_h(c->nops);
    if (!c->cu(cudaMemcpyAsync(st_h.data(), c->d_status, sizeof(int) * c->nops, cudaMemcpyDeviceToHost, c->st),
               "coarse status") ||
        !c->cu(cudaStreamSynchronize(c->st), "coarse setup"))
      return PINT_ERR_CUDA;
    for (int o = 0; o < c->nops; ++o)
      if (st_h[o] != 0) return c->fail(PINT_ERR_ARG, "coarse-grid operator is singular or too large");
  }
  return PINT_OK;
}

pint_status build(pint_ctx* c) {
  const pint_params& p = c->p;
  c->N = 1 << p.level;
  c->K = p.n_t;
  c->J = c->role == 2 ? c->role_cap : p.n_t / 2 + 1;
  c->nlev = p.level;  // grids N, N/2, ..., 2
  c->oseen = p.kind == PINT_OSEEN;
  c->conv = p.wind != PINT_WIND_NONE;
  c->gwind = p.wind == PINT_WIND_TWO_VORTEX || p.wind == PINT_WIND_NODAL;
  c->fp32 = p.prec == PINT_PREC_FP32;
  c->omega_conv = p.sor_omega_conv > 0 ? p.sor_omega_conv : p.sor_omega;
  c->m_in = p.fixed_inner_its > 0 ? p.fixed_inner_its : p.inner_maxit;
  const int N = c->N, J = c->J;
  Slots& s = c->s;
  s.n2 = 2 * N + 1;
  s.n1 = N + 1;
  s.ns = s.n2 * s.n2;
  s.nq = s.n1 * s.n1;
  s.vx = 0;
  s.vy = s.ns;
  s.p = 2LL * s.ns;
  s.lx = 2LL * s.ns + s.nq;
  s.ly = 3LL * s.ns + s.nq;
  s.mu = 4LL * s.ns + s.nq;
  s.nblk = 4LL * s.ns + 2LL * s.nq;

  if (!c->cu(cudaStreamSynchronize(c->st), "stream check")) return PINT_ERR_CUDA;
  if (!c->cu(cudaStreamCreateWithFlags(&c->st_aux, cudaStreamNonBlocking), "second stream") ||
      !c->cu(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "fork event") ||
      !c->cu(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "join event"))
    return PINT_ERR_CUDA;

  // ---- 1-D band tables per level, FP64 and FP32
  c->t64.nlev = c->t32.nlev = c->nlev;
  for (int l = 0; l < c->nlev; ++l) {
    const int Nl = N >> l;
    std::vector<double> q2, q1;
    build_level_tables(Nl, p.x0, p.x1, q2, q1);
    std::vector<float> q2f(q2.begin(), q2.end()), q1f(q1.begin(), q1.end());
    double *d2, *d1;
    float *f2, *f1;
    if (!c->upload(&d2, q2) || !c->upload(&d1, q1) || !c->upload(&f2, q2f) || !c->upload(&f1, q1f))
      return c->fail(PINT_ERR_OOM, "device allocation failed (tables)");
    c->t64.N[l] = c->t32.N[l] = Nl;
    c->t64.q2[l] = d2;
    c->t64.q1[l] = d1;
    c->t32.q2[l] = f2;
    c->t32.q1[l] = f1;
  }
  {
    std::vector<double> bt;
    build_b_tables(N, p.x0, p.x1, bt);
    std::vector<float> btf(bt.begin(), bt.end());
    double* d;
    float* f;
    if (!c->upload(&d, bt) || !c->upload(&f, btf)) return c->fail(PINT_ERR_OOM, "device allocation failed (B)");
    c->t64.bt = d;
    c->t32.bt = f;
  }
  // ---- convection stencils of the two-vortex wind (Sec. 5.2) or of a nodal
  // wind (its values injected to each coarser grid), every level
  if (c->gwind)
    for (int l = 0; l < c->nlev; ++l) {
      std::vector<double> q2, q1;
      level_convection_stencils(p, c->wind_nodal.data(), l, q2, q1);
      if (!c->upload(&c->nst64[l], q2) || (l == 0 && !c->upload(&c->npst64, q1)))
        return c->fail(PINT_ERR_OOM, "device allocation failed (convection stencils)");
    }

  // ---- per-frequency tables and job tables (Sec. 3.1-3.2, Sec. 4); a shared
  // context fills them per batch, a member has none
  if (c->role != 1) {
    if (!alloc_freq_tables(c, J)) return c->fail(PINT_ERR_OOM, "device allocation failed (frequency tables)");
    if (c->role == 0) {
      std::vector<FreqDesc> fd(J);
      for (int j = 0; j < J; ++j) fd[j] = FreqDesc{p.tau, p.beta, c->K, j};
      const pint_status rc = fill_freq_tables(c, fd);
      if (rc != PINT_OK) return rc;
    }
  }
  bool ok = true;

  // ---- multigrid / Chebyshev workspaces
  c->lay2 = make_layout(c->nlev, N, 2);
  c->lay1 = make_layout(c->nlev, N, 1);
  c->cheb_per_q2 = 2LL * s.ns;
  c->cheb_per_q1 = 2LL * s.nq;
  // workspace slots: jobs x 2 fields per job
  const size_t mgq2 = c->oseen ? 2 * (size_t)J : 4 * (size_t)J;
  const size_t mgq1 = 2 * (size_t)J;
  const size_t chq2 = c->oseen ? 2 * (size_t)J : 2;
  const size_t chq1 = 2 * (size_t)J;

  // ---- inner GMRES state
  if (!p.linear && c->role != 1) {
    GmresState& G = c->gs;
    G.J = J;
    G.m = c->m_in;
    const size_t m = (size_t)c->m_in;
    ok = c->alloc(&G.H, sizeof(double) * 2 * J * (m + 1) * m) && c->alloc(&G.g, sizeof(double) * 2 * J * (m + 1)) &&
         c->alloc(&G.cs, sizeof(double) * J * m) && c->alloc(&G.sn, sizeof(double) * 2 * J * m) &&
         c->alloc(&G.beta0, sizeof(double) * J) && c->alloc(&G.y, sizeof(double) * 2 * J * m) &&
         c->alloc(&G.partial, sizeof(double) * 2 * J * GM_CH) && c->alloc(&G.active, sizeof(int) * J) &&
         c->alloc(&G.its, sizeof(int) * J) && c->alloc(&G.count, sizeof(int)) &&
         c->alloc(&G.hc, sizeof(double) * 2 * 128 * J) && c->alloc(&G.hc2, sizeof(double) * 2 * 128 * J) &&
         c->alloc(&G.npart, sizeof(double) * GM_CH * J) &&
         c->alloc(&G.cpart, sizeof(double) * 2 * GM_CH * J * (m + 1));
    if (!ok) return c->fail(PINT_ERR_OOM, "device allocation failed (inner GMRES)");
  }
  if (c->fp32)
    ok = setup_engine<float>(c, c->e32, mgq2, mgq1, chq2, chq1);
  else
    ok = setup_engine<double>(c, c->e64, mgq2, mgq1, chq2, chq1);
  if (!ok) return c->fail(PINT_ERR_OOM, "device allocation failed (preconditioner workspace)");
  if (c->role == 2) {
    // shared frequency-domain context: no DFT, no outer FGMRES
    if (!c->cu(cudaMallocHost(&c->h_count, sizeof(int)), "pinned host buffer")) return PINT_ERR_OOM;
    if (!c->cu(cudaStreamSynchronize(c->st), "setup")) return PINT_ERR_CUDA;
    return PINT_OK;
  }
  {
    const int mode = p.dft_mode == PINT_DFT_AUTO ? (c->fp32 && c->K <= 256 ? PINT_DFT_BF16X6 : PINT_DFT_SIMT)
                                                 : p.dft_mode;
    if (mode == PINT_DFT_BF16X6 || mode == PINT_DFT_TF32X3) {
      DftTc& d = c->tc;
      dft_tc_geometry(c->K, mode == PINT_DFT_BF16X6 ? DFT_TC_BF16X6 : DFT_TC_TF32X3, &d);
      std::vector<unsigned char> tf(dft_tc_table_bytes(c->K, d.scheme, false)),
          ti(dft_tc_table_bytes(c->K, d.scheme, true));
      dft_tc_build_table(c->K, d.scheme, false, tf.data());
      dft_tc_build_table(c->K, d.scheme, true, ti.data());
      unsigned char *bf = nullptr, *bi = nullptr;
      if (!c->upload(&bf, tf) || !c->upload(&bi, ti) || !c->alloc(&d.err, sizeof(int)))
        return c->fail(PINT_ERR_OOM, "device allocation failed (DFT tables)");
      d.bf = bf;
      d.bi = bi;
      if (!c->cu(cudaMemsetAsync(d.err, 0, sizeof(int), c->st), "DFT error flag") ||
          !c->cu(cudaMallocHost(&c->h_tcerr, sizeof(int)), "pinned host buffer"))
        return PINT_ERR_CUDA;
    }
  }

  // ---- outer FGMRES workspace (FP64)
  const size_t n = (size_t)c->K * s.nblk;
  const size_t m = (size_t)p.outer_restart;
  ok = c->alloc(&c->oV, sizeof(double) * n * (m + 1)) && c->alloc(&c->oZ, sizeof(double) * n * m) &&
       c->alloc(&c->ob, sizeof(double) * n) && c->alloc(&c->ox, sizeof(double) * n) &&
       c->alloc(&c->ot, sizeof(double) * n) && c->alloc(&c->opart, sizeof(double) * MDOT_CTAS * 8) &&
       c->alloc(&c->oh, sizeof(double) * (2 * m + 8)) &&
       c->alloc(&c->ofreq, sizeof(double) * 2 * (size_t)J * s.nblk);
  if (!ok) return c->fail(PINT_ERR_OOM, "device allocation failed (outer FGMRES)");
  if (!c->cu(cudaMallocHost(&c->h_pinned, sizeof(double) * (2 * m + 8)), "pinned host buffer") ||
      !c->cu(cudaMallocHost(&c->h_count, sizeof(int)), "pinned host buffer"))
    return PINT_ERR_OOM;
  if (!c->cu(cudaStreamSynchronize(c->st), "setup")) return PINT_ERR_CUDA;
  return PINT_OK;
}

// Reads (and clears) the tensor-core DFT's device error flag: nonzero means a
// bounded wait inside the kernel gave up and its output is not valid.
pint_status tc_status(pint_ctx* c) {
  if (!c->tc.scheme) return PINT_OK;
  if (!c->cu(cudaMemcpyAsync(c->h_tcerr, c->tc.err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "DFT status") ||
      !c->cu(cudaStreamSynchronize(c->st), "DFT status"))
    return PINT_ERR_CUDA;
  if (*c->h_tcerr == 0) return PINT_OK;
  cudaMemsetAsync(c->tc.err, 0, sizeof(int), c->st);
  return c->fail(PINT_ERR_TIMEOUT, "tensor-core DFT: a bounded wait gave up; results are not valid");
}

void free_ctx(pint_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->st_aux) {
    cudaStreamSynchronize(c->st_aux);
    cudaStreamDestroy(c->st_aux);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  c->drain();
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  for (void* v : c->allocs) cudaFree(v);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->h_count) cudaFreeHost(c->h_count);
  if (c->h_tcerr) cudaFreeHost(c->h_tcerr);
  delete c;
}

// ---------------------------------------------------------------- wrappers
void kkt(pint_ctx* c, const double* x, double* y) {
  KKTArgs a{};
  a.tabs = c->t64;
  a.s = c->s;
  a.K = c->K;
  a.tau = c->p.tau;
  a.beta = c->p.beta;
  a.nu = c->p.nu;
  a.conv = c->conv && !c->gwind;
  a.nst = c->gwind ? c->nst64[0] : nullptr;
  a.x = x;
  a.y = y;
  c->add_bytes(PINT_PROF_KKT_MV, 16.0 * c->K * c->s.nblk);
  PROF(c, PINT_PROF_KKT_MV, 2);
  launch_kkt_matvec(a, c->st);
}

void apply_prec(pint_ctx* c, const double* r, double* z, int* its) {
  PROF(c, PINT_PROF_APPLY, 0);
  if (c->fp32)
    c->e32.apply(r, z, its);
  else
    c->e64.apply(r, z, its);
}

inline int mdot_kernels(int cnt) { return 2 * ((cnt + 7) / 8); }

double dot_dev(pint_ctx* c, const double* a, const double* b, long long n) {
  c->add_bytes(PINT_PROF_OUTER, (a == b ? 8.0 : 16.0) * n);
  {
    PROF(c, PINT_PROF_OUTER, mdot_kernels(1));
    launch_mdot(a, 1, b, n, c->opart, c->oh, c->st);
  }
  cudaMemcpyAsync(c->h_pinned, c->oh, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  cudaStreamSynchronize(c->st);
  return c->h_pinned[0];
}

// Outer FP64 FGMRES(m) with classical Gram-Schmidt + reorthogonalisation.
pint_status fgmres(pint_ctx* c, double* x, pint_solve_info* info) {
  const long long n = (long long)c->K * c->s.nblk;
  const int m = c->p.outer_restart;
  cudaStream_t st = c->st;
  pint_solve_info inf{};
  const auto t0 = std::chrono::steady_clock::now();
  double t_prec = 0, t_mv = 0, t_orth = 0;
  auto now = [] { return std::chrono::steady_clock::now(); };
  auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  std::vector<int> its(c->J, 0);
  const double bnorm = std::sqrt(dot_dev(c, c->ob, c->ob, n));
  if (bnorm == 0.0) {
    cudaMemsetAsync(x, 0, sizeof(double) * n, st);
    cudaStreamSynchronize(st);
    if (info) *info = inf;
    return PINT_OK;
  }
  // r = b - A x
  kkt(c, x, c->ot);
  c->add_bytes(PINT_PROF_OUTER, 24.0 * n);
  {
    PROF(c, PINT_PROF_OUTER, 1);
    launch_axpby(1.0, c->ob, -1.0, c->ot, n, st);
  }
  double beta = std::sqrt(dot_dev(c, c->ot, c->ot, n));
  double relres = beta / bnorm;
  int total = 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  while (total < c->p.outer_maxit && relres > c->p.outer_tol) {
    c->add_bytes(PINT_PROF_OUTER, 16.0 * n);
    {
      PROF(c, PINT_PROF_OUTER, 1);
      launch_axpby(1.0 / beta, c->ot, 0.0, c->oV, n, st);
    }
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int i = 0; i < m; ++i) {
      double* Vi = c->oV + (size_t)i * n;
      double* Zi = c->oZ + (size_t)i * n;
      double* Vn = c->oV + (size_t)(i + 1) * n;
      auto a0 = now();
      apply_prec(c, Vi, Zi, its.data());
      cudaStreamSynchronize(st);
      ++c->prof_syncs;
      if (c->batch_rc != PINT_OK) {
        inf.outer_iterations = total;
        if (info) *info = inf;
        return c->batch_rc;
      }
      auto a1 = now();
      for (int j = 0; j < c->J; ++j) {
        inf.inner_iterations_total += its[j];
        inf.inner_iterations_max = std::max(inf.inner_iterations_max, its[j]);
      }
      inf.precond_applies++;
      kkt(c, Zi, Vn);
      cudaStreamSynchronize(st);
      auto a2 = now();
      // CGS2
      c->add_bytes(PINT_PROF_OUTER, (4.0 * i + 11.0) * 8.0 * n);
      {
        PROF(c, PINT_PROF_OUTER, 2 * mdot_kernels(i + 1) + 2 + mdot_kernels(1));
      launch_mdot(c->oV, i + 1, Vn, n, c->opart, c->oh, st);
      launch_maxpy(c->oV, i + 1, c->oh, Vn, n, st);
      launch_mdot(c->oV, i + 1, Vn, n, c->opart, c->oh + (i + 1), st);
      launch_maxpy(c->oV, i + 1, c->oh + (i + 1), Vn, n, st);
      launch_mdot(Vn, 1, Vn, n, c->opart, c->oh + 2 * (i + 1), st);
      }
      cudaMemcpyAsync(c->h_pinned, c->oh, sizeof(double) * (2 * (i + 1) + 1), cudaMemcpyDeviceToHost, st);
      if (!c->cu(cudaStreamSynchronize(st), "FGMRES iteration")) return PINT_ERR_CUDA;
      ++c->prof_syncs;
      c->drain();
      for (int l = 0; l <= 2 * (i + 1); ++l)
        if (!std::isfinite(c->h_pinned[l])) {
          inf.outer_iterations = total;
          inf.relres = NAN;
          if (info) *info = inf;
          return c->fail(PINT_ERR_NONFINITE, "non-finite value in the preconditioned Krylov vector (iteration " +
                                                 std::to_string(total + 1) + ")");
        }
      const double hn = std::sqrt(std::max(0.0, c->h_pinned[2 * (i + 1)]));
      for (int l = 0; l <= i; ++l) H[(size_t)l * m + i] = c->h_pinned[l] + c->h_pinned[i + 1 + l];
      H[(size_t)(i + 1) * m + i] = hn;
      if (hn != 0.0) {
        c->add_bytes(PINT_PROF_OUTER, 16.0 * n);
        PROF(c, PINT_PROF_OUTER, 1);
        launch_axpby(1.0 / hn, Vn, 0.0, Vn, n, st);
      }
      auto a3 = now();
      t_prec += ms(a0, a1);
      t_mv += ms(a1, a2);
      t_orth += ms(a2, a3);
      for (int l = 0; l < i; ++l) {
        const double t = cs[l] * H[(size_t)l * m + i] + sn[l] * H[(size_t)(l + 1) * m + i];
        H[(size_t)(l + 1) * m + i] = -sn[l] * H[(size_t)l * m + i] + cs[l] * H[(size_t)(l + 1) * m + i];
        H[(size_t)l * m + i] = t;
      }
      const double den = std::hypot(H[(size_t)i * m + i], hn);
      cs[i] = H[(size_t)i * m + i] / den;
      sn[i] = hn / den;
      H[(size_t)i * m + i] = den;
      H[(size_t)(i + 1) * m + i] = 0.0;
      g[i + 1] = -sn[i] * g[i];
      g[i] = cs[i] * g[i];
      ++total;
      k = i + 1;
      if (total <= 256) inf.relres_history[total - 1] = std::fabs(g[i + 1]) / bnorm;
      if (std::fabs(g[i + 1]) <= c->p.outer_tol * bnorm || total >= c->p.outer_maxit || hn == 0.0) break;
    }
    for (int l = k - 1; l >= 0; --l) {
      double sacc = g[l];
      for (int q = l + 1; q < k; ++q) sacc -= H[(size_t)l * m + q] * y[q];
      y[l] = sacc / H[(size_t)l * m + l];
    }
    for (int l = 0; l < k; ++l) c->h_pinned[l] = -y[l];
    cudaMemcpyAsync(c->oh, c->h_pinned, sizeof(double) * k, cudaMemcpyHostToDevice, st);
    c->add_bytes(PINT_PROF_OUTER, (k + 2.0) * 8.0 * n);
    {
      PROF(c, PINT_PROF_OUTER, 1);
      launch_maxpy(c->oZ, k, c->oh, x, n, st);  // x += Z y
    }
    kkt(c, x, c->ot);
    c->add_bytes(PINT_PROF_OUTER, 24.0 * n);
    {
      PROF(c, PINT_PROF_OUTER, 1);
      launch_axpby(1.0, c->ob, -1.0, c->ot, n, st);
    }
    beta = std::sqrt(dot_dev(c, c->ot, c->ot, n));
    relres = beta / bnorm;
    inf.restarts++;
    if (!c->launched("FGMRES restart")) return PINT_ERR_CUDA;
  }
  inf.outer_iterations = total;
  inf.relres = relres;
  inf.ms_precond = t_prec;
  inf.ms_matvec = t_mv;
  inf.ms_orth = t_orth;
  inf.ms_total = ms(t0, now());
  if (info) *info = inf;
  return relres <= c->p.outer_tol ? PINT_OK : c->fail(PINT_ERR_NOT_CONVERGED, "outer FGMRES did not converge");
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void pint_default_params(pint_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->kind = PINT_STOKES;
  p->level = 3;
  p->x0 = 0.0;
  p->x1 = 1.0;
  p->n_t = 8;
  p->tau = 1.0 / 9.0;
  p->beta = 1e-2;
  p->nu = 1e-2;
  p->wind = PINT_WIND_NONE;
  p->prec = PINT_PREC_FP64;
  p->outer_restart = 30;
  p->outer_maxit = 300;
  p->outer_tol = 1e-8;
  p->inner_tol = 1e-2;
  p->inner_maxit = 100;
  p->mg_cycles = 4;
  p->mg_pre = 2;
  p->mg_post = 2;
  p->cheb_steps = 10;
  p->uzawa_steps = 6;
  p->uzawa_mu = 0.75;
  p->sor_omega = 1.0;
  p->fixed_inner_its = 0;
  p->linear = 0;
  p->dft_mode = PINT_DFT_AUTO;
  p->sor_omega_conv = 0.0;
}

size_t pint_estimate_device_bytes(const pint_params* p) {
  std::string why;
  if (!valid_params(p, why)) return 0;
  const long long N = 1LL << p->level, K = p->n_t, J = K / 2 + 1;
  const long long ns = (2 * N + 1) * (2 * N + 1), nq = (N + 1) * (N + 1), nblk = 4 * ns + 2 * nq;
  const bool fp32 = p->prec == PINT_PREC_FP32, oseen = p->kind == PINT_OSEEN;
  const long long cs = fp32 ? 8 : 16;  // bytes per complex value of the preconditioner
  const long long m = p->outer_restart;
  const long long m_in = p->fixed_inner_its > 0 ? p->fixed_inner_its : p->inner_maxit;
  long long b = 0;
  b += (2 * m + 4) * K * nblk * 8 + J * nblk * 16;  // outer FGMRES basis, b, x, t; FP64 frequency staging
  b += 5 * J * nblk * cs;                            // frequency vectors
  if (!p->linear) b += (2 * m_in + 1) * J * nblk * cs + (long long)J * (m_in + 1) * m_in * 16 * 2;
  const MGLayout l2 = make_layout(p->level, (int)N, 2), l1 = make_layout(p->level, (int)N, 1);
  const long long mgq2 = oseen ? 2 * J : 4 * J, mgq1 = 2 * J, chq2 = oseen ? 2 * J : 2, chq1 = 2 * J;
  b += std::max(mgq2 * l2.per_job, mgq1 * l1.per_job) * cs;
  if (!oseen) b += mgq1 * l1.per_job * cs;  // pressure multigrid beside the velocity one
  b += std::max(chq2 * 2 * ns, chq1 * 2 * nq) * cs;
  if (p->wind != PINT_WIND_NONE)
    for (int l = 0; l < p->level; ++l) {
      const long long n2 = 2 * (N >> l) + 1, w6 = (n2 + 5) / 6;
      b += 36 * w6 * w6 * 25 * (fp32 ? 4 : 8) + nq * 9 * 8;
      if (p->wind == PINT_WIND_TWO_VORTEX || p->wind == PINT_WIND_NODAL)
        b += n2 * n2 * 25 * 8 + (l == 0 ? nq * 9 * 8 : 0);
    }
  return (size_t)(b + b / 20 + (64LL << 20));  // 5% + 64 MiB for tables and small state
}

namespace {

pint_status create_impl(const pint_params* p, const double* wind, void* stream, pint_handle* out) {
  if (!out) {
    g_err = "null output handle";
    return PINT_ERR_ARG;
  }
  *out = nullptr;
  std::string why;
  if (!valid_params(p, why)) {
    g_err = why;
    return PINT_ERR_ARG;
  }
  if ((p->wind == PINT_WIND_NODAL) != (wind != nullptr)) {
    g_err = wind ? "a nodal wind needs p->wind = PINT_WIND_NODAL"
                 : "PINT_WIND_NODAL needs the wind's nodal values (pint_create_wind)";
    return PINT_ERR_ARG;
  }
  const size_t nw = wind ? 2 * (size_t)((2 << p->level) + 1) * ((2 << p->level) + 1) : 0;
  for (size_t i = 0; i < nw; ++i)
    if (!std::isfinite(wind[i])) {
      g_err = "non-finite value in the nodal wind";
      return PINT_ERR_NONFINITE;
    }
  pint_ctx* c = new (std::nothrow) pint_ctx();
  if (!c) {
    g_err = "host allocation failed";
    return PINT_ERR_OOM;
  }
  c->p = *p;
  c->st = static_cast<cudaStream_t>(stream);
  if (wind) c->wind_nodal.assign(wind, wind + nw);
  pint_status s = build(c);
  if (s != PINT_OK) {
    std::string m = c->err;
    free_ctx(c);
    g_err = m;
    return s;
  }
  *out = c;
  return PINT_OK;
}

}  // namespace

pint_status pint_create(const pint_params* p, void* stream, pint_handle* out) {
  return create_impl(p, nullptr, stream, out);
}

pint_status pint_create_wind(const pint_params* p, const double* wind_host, void* stream, pint_handle* out) {
  if (!wind_host) {
    g_err = "wind_host must not be null";
    return PINT_ERR_ARG;
  }
  return create_impl(p, wind_host, stream, out);
}

pint_status pint_convection_stencils(const pint_params* p, const double* wind_host, int l, double* q2_out,
                                     double* q1_out) {
  std::string why;
  if (!valid_params(p, why)) {
    g_err = why;
    return PINT_ERR_ARG;
  }
  if (p->wind != PINT_WIND_TWO_VORTEX && p->wind != PINT_WIND_NODAL) {
    g_err = "stencils exist for PINT_WIND_TWO_VORTEX and PINT_WIND_NODAL only";
    return PINT_ERR_ARG;
  }
  if ((p->wind == PINT_WIND_NODAL) != (wind_host != nullptr) || l < 0 || l >= p->level) {
    g_err = "wind_host must be given exactly for PINT_WIND_NODAL, and 0 <= l < level";
    return PINT_ERR_ARG;
  }
  std::vector<double> q2, q1;
  level_convection_stencils(*p, wind_host, l, q2, q1);
  if (q2_out) std::memcpy(q2_out, q2.data(), q2.size() * sizeof(double));
  if (q1_out) std::memcpy(q1_out, q1.data(), q1.size() * sizeof(double));
  return PINT_OK;
}

void member_destroy(pint_handle h);

pint_status pint_destroy(pint_handle h) {
  if (h && h->role == 1)
    member_destroy(h);
  else
    free_ctx(h);
  return PINT_OK;
}

pint_status pint_get_sizes(pint_handle h, pint_sizes* s) {
  if (!h || !s) {
    g_err = "null argument";
    return PINT_ERR_ARG;
  }
  s->N = h->N;
  s->n_t = h->K;
  s->J = h->J;
  s->n_s = (size_t)h->s.ns;
  s->n_q = (size_t)h->s.nq;
  s->n_blk = (size_t)h->s.nblk;
  s->kkt_len = (size_t)h->K * h->s.nblk;
  s->freq_len = (size_t)h->J * h->s.nblk;
  s->device_bytes = h->dev_bytes;
  return PINT_OK;
}

namespace {

// Uploads the problem data and builds b on the device.  full = 0: loads from
// interior nodal values only (pint_set_data).  full = 1: loads from every
// nodal value, and the known boundary velocity g (may be null) is lifted to
// the right-hand side as b -= A x_g, where x_g holds g_k in the boundary
// entries of the state-velocity slots; A x_g is the Eq. FinalA matvec on the
// whole grid, read at the interior rows (pint_set_data_dirichlet).
pint_status set_data_impl(pint_handle h, const double* vd, const double* f, const double* v0, const double* g,
                          int full) {
  if (!h) {
    g_err = "null handle";
    return PINT_ERR_ARG;
  }
  if (!vd) return h->fail(PINT_ERR_ARG, "vd must not be null");
  const size_t nvd = (size_t)h->K * 2 * h->s.ns, nv0 = 2 * (size_t)h->s.ns;
  for (size_t i = 0; i < nvd; ++i)
    if (!std::isfinite(vd[i]) || (f && !std::isfinite(f[i])) || (g && !std::isfinite(g[i])))
      return h->fail(PINT_ERR_NONFINITE, "non-finite value in vd, f or g");
  if (v0)
    for (size_t i = 0; i < nv0; ++i)
      if (!std::isfinite(v0[i])) return h->fail(PINT_ERR_NONFINITE, "non-finite value in v0");
  const size_t nkkt = (size_t)h->K * h->s.nblk;
  double *dvd = nullptr, *df = nullptr, *dv0 = nullptr, *dg = nullptr, *dxg = nullptr, *dyg = nullptr;
  bool ok = cudaMalloc(&dvd, sizeof(double) * nvd) == cudaSuccess;
  if (ok && f) ok = cudaMalloc(&df, sizeof(double) * nvd) == cudaSuccess;
  if (ok && v0) ok = cudaMalloc(&dv0, sizeof(double) * nv0) == cudaSuccess;
  if (ok && g) ok = cudaMalloc(&dg, sizeof(double) * nvd) == cudaSuccess;
  if (ok && g) ok = cudaMalloc(&dxg, sizeof(double) * nkkt) == cudaSuccess;
  if (ok && g) ok = cudaMalloc(&dyg, sizeof(double) * nkkt) == cudaSuccess;
  pint_status rc = PINT_OK;
  if (!ok) {
    cudaGetLastError();
    rc = h->fail(PINT_ERR_OOM, "device allocation failed (data)");
  } else {
    ok = h->cu(cudaMemcpy(dvd, vd, sizeof(double) * nvd, cudaMemcpyHostToDevice), "upload vd");
    if (ok && f) ok = h->cu(cudaMemcpy(df, f, sizeof(double) * nvd, cudaMemcpyHostToDevice), "upload f");
    if (ok && v0) ok = h->cu(cudaMemcpy(dv0, v0, sizeof(double) * nv0, cudaMemcpyHostToDevice), "upload v0");
    if (ok && g) ok = h->cu(cudaMemcpy(dg, g, sizeof(double) * nvd, cudaMemcpyHostToDevice), "upload g");
    if (ok) {
      RhsArgs a{};
      a.tabs = h->t64;
      a.s = h->s;
      a.K = h->K;
      a.tau = h->p.tau;
      a.vd = dvd;
      a.f = df;
      a.v0 = dv0;
      a.b = h->ob;
      a.full = full;
      launch_rhs(a, h->st);
      ok = h->launched("rhs");
    }
    if (ok && g) {
      ok = h->cu(cudaMemsetAsync(dxg, 0, sizeof(double) * nkkt, h->st), "clear lift");
      if (ok) {
        launch_lift_scatter(h->s, h->K, dg, dxg, h->st);
        kkt(h, dxg, dyg);
        launch_axpby(-1.0, dyg, 1.0, h->ob, (long long)nkkt, h->st);
        ok = h->launched("lift");
      }
    }
    if (ok) ok = h->cu(cudaStreamSynchronize(h->st), "rhs");
    if (!ok) rc = PINT_ERR_CUDA;
  }
  cudaFree(dvd);
  if (df) cudaFree(df);
  if (dv0) cudaFree(dv0);
  if (dg) cudaFree(dg);
  if (dxg) cudaFree(dxg);
  if (dyg) cudaFree(dyg);
  if (rc == PINT_OK) h->have_data = true;
  return rc;
}

}  // namespace

pint_status pint_set_data(pint_handle h, const double* vd, const double* f, const double* v0) {
  return set_data_impl(h, vd, f, v0, nullptr, 0);
}

pint_status pint_set_data_dirichlet(pint_handle h, const double* vd, const double* f, const double* v0,
                                    const double* g) {
  return set_data_impl(h, vd, f, v0, g, 1);
}

pint_status pint_get_rhs(pint_handle h, double* b_dev) {
  if (!h || !b_dev) {
    g_err = "null argument";
    return PINT_ERR_ARG;
  }
  if (!h->have_data) return h->fail(PINT_ERR_STATE, "pint_set_data has not been called");
  const size_t n = (size_t)h->K * h->s.nblk;
  if (!h->cu(cudaMemcpyAsync(b_dev, h->ob, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "copy rhs"))
    return PINT_ERR_CUDA;
  return PINT_OK;
}

pint_status pint_kkt_matvec(pint_handle h, const double* x, double* y) {
  if (!h || !x || !y) {
    g_err = "null argument";
    return PINT_ERR_ARG;
  }
  const size_t n = (size_t)h->K * h->s.nblk;
  if (!h->cu(cudaMemcpyAsync(h->ox, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "copy x"))
    return PINT_ERR_CUDA;
  { PROF(h, PINT_PROF_OTHER, 1); launch_mask_blocks(h->s, h->K, 1, h->ox, h->st); }
  kkt(h, h->ox, y);
  return h->launched("kkt matvec") ? PINT_OK : PINT_ERR_CUDA;
}

pint_status pint_apply_preconditioner(pint_handle h, const double* r, double* z) {
  if (!h || !r || !z) {
    g_err = "null argument";
    return PINT_ERR_ARG;
  }
  const size_t n = (size_t)h->K * h->s.nblk;
  if (!h->cu(cudaMemcpyAsync(h->ot, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "copy r"))
    return PINT_ERR_CUDA;
  { PROF(h, PINT_PROF_OTHER, 1); launch_mask_blocks(h->s, h->K, 1, h->ot, h->st); }
  apply_prec(h, h->ot, z, nullptr);
  if (!h->launched("preconditioner")) return PINT_ERR_CUDA;
  return tc_status(h);
}

}  // extern "C"
static void member_solve_begin(pint_handle h);
static void member_solve_end(pint_handle h);
extern "C" {

pint_status pint_solve(pint_handle h, double* x, pint_solve_info* info) {
  if (!h || !x) {
    g_err = "null argument";
    return PINT_ERR_ARG;
  }
  if (!h->have_data) return h->fail(PINT_ERR_STATE, "pint_set_data has not been called");
  const size_t n = (size_t)h->K * h->s.nblk;
  if (!h->cu(cudaMemcpyAsync(h->ox, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "copy x0"))
    return PINT_ERR_CUDA;
  { PROF(h, PINT_PROF_OTHER, 1); launch_mask_blocks(h->s, h->K, 1, h->ox, h->st); }
  if (h->role == 1) member_solve_begin(h);
  pint_status rc = fgmres(h, h->ox, info);
  if (h->role == 1) member_solve_end(h);
  if (!h->cu(cudaMemcpyAsync(x, h->ox, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st), "copy x") ||
      !h->cu(cudaStreamSynchronize(h->st), "solve"))
    return PINT_ERR_CUDA;
  const pint_status ts = tc_status(h);
  return ts != PINT_OK ? ts : rc;
}

pint_status pint_solve_host(pint_handle h, double* x_host, pint_solve_info* info) {
  if (!h || !x_host) {
    g_err = "null argument";
    return PINT_ERR_ARG;
  }
  if (!h->have_data) return h->fail(PINT_ERR_STATE, "pint_set_data has not been called");
  const size_t n = (size_t)h->K * h->s.nblk;
  if (!h->cu(cudaMemcpyAsync(h->ox, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->st), "upload x0"))
    return PINT_ERR_CUDA;
  { PROF(h, PINT_PROF_OTHER, 1); launch_mask_blocks(h->s, h->K, 1, h->ox, h->st); }
  if (h->role == 1) member_solve_begin(h);
  pint_status rc = fgmres(h, h->ox, info);
  if (h->role == 1) member_solve_end(h);
  if (!h->cu(cudaMemcpyAsync(x_host, h->ox, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st), "download x") ||
      !h->cu(cudaStreamSynchronize(h->st), "solve"))
    return PINT_ERR_CUDA;
  const pint_status ts = tc_status(h);
  return ts != PINT_OK ? ts : rc;
}

}  // extern "C"

// -------------------------------------------------------- component entries
namespace {
template <class T>
void to_T(pint_ctx* c, const double* src, cpx<T>* dst, size_t ncplx);
template <>
void to_T<double>(pint_ctx* c, const double* src, cpx<double>* dst, size_t n) {
  cudaMemcpyAsync(dst, src, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, c->st);
}
template <>
void to_T<float>(pint_ctx* c, const double* src, cpx<float>* dst, size_t n) {
  launch_copy_d2f(src, reinterpret_cast<float*>(dst), (long long)(2 * n), c->st);
}
template <class T>
void from_T(pint_ctx* c, const cpx<T>* src, double* dst, size_t ncplx);
template <>
void from_T<double>(pint_ctx* c, const cpx<double>* src, double* dst, size_t n) {
  cudaMemcpyAsync(dst, src, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, c->st);
}
template <>
void from_T<float>(pint_ctx* c, const cpx<float>* src, double* dst, size_t n) {
  launch_copy_f2d(reinterpret_cast<const float*>(src), dst, (long long)(2 * n), c->st);
}

template <class T>
pint_status dft_fwd_T(pint_ctx* c, Engine<T>& e, const double* x, double* xhat) {
  const size_t n = (size_t)c->K * c->s.nblk;
  cudaMemcpyAsync(c->ot, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st);
  { PROF(c, PINT_PROF_OTHER, 1); launch_mask_blocks(c->s, c->K, 1, c->ot, c->st); }
  dft_forward_any<T>(c, e, c->ot, e.R);
  from_T<T>(c, e.R, xhat, (size_t)c->J * c->s.nblk);
  if (!c->launched("dft forward")) return PINT_ERR_CUDA;
  return tc_status(c);
}

template <class T>
pint_status dft_inv_T(pint_ctx* c, Engine<T>& e, const double* xhat, double* x) {
  const size_t fl = (size_t)c->J * c->s.nblk;
  to_T<T>(c, xhat, e.R, fl);
  dft_inverse_any<T>(c, e, e.R, x);
  { PROF(c, PINT_PROF_OTHER, 1); launch_mask_blocks(c->s, c->K, 1, x, c->st); }
  if (!c->launched("dft inverse")) return PINT_ERR_CUDA;
  return tc_status(c);
}

template <class T>
pint_status freq_in(pint_ctx* c, Engine<T>& e, const double* in) {
  // copy, zero the non-unknown entries in FP64, then convert to T
  const size_t fl = (size_t)c->J * c->s.nblk;
  cudaMemcpyAsync(c->ofreq, in, sizeof(double) * 2 * fl, cudaMemcpyDeviceToDevice, c->st);
  { PROF(c, PINT_PROF_OTHER, 1); launch_mask_blocks(c->s, c->J, 2, c->ofreq, c->st); }
  to_T<T>(c, c->ofreq, e.R, fl);
  return PINT_OK;
}

template <class T>
pint_status block_mv_T(pint_ctx* c, Engine<T>& e, const double* in, double* out) {
  const size_t fl = (size_t)c->J * c->s.nblk;
  freq_in<T>(c, e, in);
  e.block_matvec(c->d_blkG, e.R, e.Y, nullptr);
  from_T<T>(c, e.Y, out, fl);
  return c->launched("block matvec") ? PINT_OK : PINT_ERR_CUDA;
}

template <class T>
pint_status block_solve_T(pint_ctx* c, Engine<T>& e, const double* in, double* out, int* its) {
  const size_t fl = (size_t)c->J * c->s.nblk;
  freq_in<T>(c, e, in);
  e.freq_solve(e.R, e.Y, its);
  from_T<T>(c, e.Y, out, fl);
  return c->launched("block solve") && c->cu(cudaStreamSynchronize(c->st), "block solve") ? PINT_OK
                                                                                          : PINT_ERR_CUDA;
}

template <class T>
pint_status component_T(pint_ctx* c, Engine<T>& e, int which, int j, const double* in, double* out) {
  const Slots& s = c->s;
  const int J = c->J;
  if (which == 6) {
    const size_t nb = (size_t)s.nblk;
    cudaMemsetAsync(e.R, 0, sizeof(cpx<T>) * J * nb, c->st);
    to_T<T>(c, in, e.R + (size_t)j * nb, nb);
    std::vector<int> act(J, 0);
    act[j] = 1;
    cudaMemcpyAsync(c->d_active_one, act.data(), sizeof(int) * J, cudaMemcpyHostToDevice, c->st);
    e.block_prec(e.R, e.Y, c->d_active_one);
    from_T<T>(c, e.Y + (size_t)j * nb, out, nb);
    return c->launched("component") && c->cu(cudaStreamSynchronize(c->st), "component") ? PINT_OK
                                                                                         : PINT_ERR_CUDA;
  }
  const int space = (which == 3 || which == 5) ? 1 : 2;
  const size_t len = space == 2 ? (size_t)s.ns : (size_t)s.nq;
  int op;
  switch (which) {
    case 0:
      if (c->oseen) return c->fail(PINT_ERR_ARG, "W_j exists for Stokes problems only");
      op = j;
      break;
    case 1:
    case 2:
      if (!c->oseen) return c->fail(PINT_ERR_ARG, "Q_j exists for Oseen problems only");
      op = which == 1 ? j : J + j;
      break;
    case 3:
      op = 2 * J;
      break;
    case 4:
      op = 2 * J + 1;
      break;
    default:
      op = 2 * J + 2;
      break;
  }
  // mask the input field on the host (diagnostic path)
  std::vector<double> hin(2 * len);
  if (!c->cu(cudaMemcpy(hin.data(), in, sizeof(double) * 2 * len, cudaMemcpyDeviceToHost), "component input"))
    return PINT_ERR_CUDA;
  const int n = space == 2 ? s.n2 : s.n1;
  for (size_t q = 0; q < len; ++q) {
    const int ix = (int)(q % n), iy = (int)(q / n);
    const bool unk = space == 2 ? (ix > 0 && iy > 0 && ix < n - 1 && iy < n - 1) : ((ix | iy) != 0);
    if (!unk) hin[2 * q] = hin[2 * q + 1] = 0.0;
  }
  double* stage = c->ot;  // FP64 scratch of kkt_len >= 2 * len doubles
  cudaMemcpyAsync(stage, hin.data(), sizeof(double) * 2 * len, cudaMemcpyHostToDevice, c->st);
  to_T<T>(c, stage, e.T1, len);
  FieldJob jb{};
  jb.nf = 1;
  jb.op = op;
  cudaMemcpyAsync(c->j_one, &jb, sizeof(FieldJob), cudaMemcpyHostToDevice, c->st);
  if (which <= 3)
    e.mg(space, which == 1 || which == 2 ? c->conv : false, c->j_one, 1, e.T2, e.T1, nullptr, 1);
  else
    e.cheb(space, c->j_one, 1, e.T2, e.T1, nullptr, 1);
  from_T<T>(c, e.T2, out, len);
  return c->launched("component") && c->cu(cudaStreamSynchronize(c->st), "component") ? PINT_OK : PINT_ERR_CUDA;
}
}  // namespace

extern "C" {

pint_status pint_dft_forward(pint_handle h, const double* x, double* xhat) {
  if (!h || !x || !xhat) return g_err = "null argument", PINT_ERR_ARG;
  return h->fp32 ? dft_fwd_T<float>(h, h->e32, x, xhat) : dft_fwd_T<double>(h, h->e64, x, xhat);
}

pint_status pint_dft_inverse(pint_handle h, const double* xhat, double* x) {
  if (!h || !x || !xhat) return g_err = "null argument", PINT_ERR_ARG;
  return h->fp32 ? dft_inv_T<float>(h, h->e32, xhat, x) : dft_inv_T<double>(h, h->e64, xhat, x);
}

pint_status pint_freq_block_matvec(pint_handle h, const double* xhat, double* yhat) {
  if (!h || !xhat || !yhat) return g_err = "null argument", PINT_ERR_ARG;
  return h->fp32 ? block_mv_T<float>(h, h->e32, xhat, yhat) : block_mv_T<double>(h, h->e64, xhat, yhat);
}

pint_status pint_freq_block_solve(pint_handle h, const double* rhat, double* yhat, int* its) {
  if (!h || !rhat || !yhat) return g_err = "null argument", PINT_ERR_ARG;
  return h->fp32 ? block_solve_T<float>(h, h->e32, rhat, yhat, its)
                 : block_solve_T<double>(h, h->e64, rhat, yhat, its);
}

pint_status pint_component_apply(pint_handle h, int which, int j, const double* in, double* out) {
  if (!h || !in || !out) return g_err = "null argument", PINT_ERR_ARG;
  if (which < 0 || which > 6) return h->fail(PINT_ERR_ARG, "which must be in [0, 6]");
  if (j < 0 || j >= h->J) return h->fail(PINT_ERR_ARG, "frequency index out of range");
  return h->fp32 ? component_T<float>(h, h->e32, which, j, in, out)
                 : component_T<double>(h, h->e64, which, j, in, out);
}

void pint_autotune(int on) { mg_autotune_enable(on != 0); }

pint_status pint_mg_launch_config(int threads, int staging) {
  if (threads != 0 && threads != 256 && threads != 512 && threads != 1024) {
    g_err = "threads must be 0, 256, 512 or 1024";
    return PINT_ERR_ARG;
  }
  if (staging < -1 || staging > 2) {
    g_err = "staging must be -1, 0, 1 or 2";
    return PINT_ERR_ARG;
  }
  mg_fixed_config(threads, staging);
  return PINT_OK;
}

size_t pint_autotune_report(char* buf, size_t len) {
  const std::string r = mg_autotune_report();
  if (buf && len) {
    const size_t n = std::min(len - 1, r.size());
    memcpy(buf, r.data(), n);
    buf[n] = 0;
  }
  return r.size() + 1;
}

pint_status pint_debug_inject(pint_handle h, int what) {
  if (!h) return g_err = "null handle", PINT_ERR_ARG;
  if (what != PINT_INJECT_DFT_STALL) return h->fail(PINT_ERR_ARG, "unknown injection code");
  if (!h->tc.scheme) return h->fail(PINT_ERR_ARG, "this handle does not use the tensor-core DFT");
  h->tc.stall_next = true;
  return PINT_OK;
}

pint_status pint_profile_enable(pint_handle h, unsigned mask) {
  if (!h) return g_err = "null handle", PINT_ERR_ARG;
  if (!h->cu(cudaStreamSynchronize(h->st), "profile enable")) return PINT_ERR_CUDA;
  h->drain();
  h->prof_mask = mask;
  for (int i = 0; i < PINT_PROF_CLASSES; ++i) {
    h->prof_launch[i] = h->prof_timed[i] = 0;
    h->prof_ms[i] = 0.0;
    h->prof_bytes[i] = 0.0;
  }
  h->prof_syncs = 0;
  return PINT_OK;
}

pint_status pint_profile_read(pint_handle h, pint_profile* out) {
  if (!h || !out) return g_err = "null argument", PINT_ERR_ARG;
  if (!h->cu(cudaStreamSynchronize(h->st), "profile read")) return PINT_ERR_CUDA;
  h->drain();
  for (int i = 0; i < PINT_PROF_CLASSES; ++i) {
    out->launches[i] = h->prof_launch[i];
    out->timed[i] = h->prof_timed[i];
    out->ms[i] = h->prof_ms[i];
    out->bytes[i] = h->prof_bytes[i];
  }
  out->host_syncs = h->prof_syncs;
  return PINT_OK;
}

const char* pint_last_error(pint_handle h) {
  if (h && !h->err.empty()) return h->err.c_str();
  return g_err.c_str();
}

}  // extern "C"

// ============================================================================
// Multigrid component solve without allocation (pint_mg_apply_noalloc).
//
// Scratch for this entry point lives in one file-scope device array instead
// of the handle's workspace: the staged input field, the output field, the
// per-level V-cycle arrays and the job descriptor.  Every GPU that loads the
// library holds the array until the process exits.  Its device address is
// looked up once per device (cudaGetSymbolAddress, with that device current)
// on the first call there; host code never hands the array's name to a
// kernel.  All calls share the array: calls that overlap on the GPU (other
// streams, other threads) race on it.
// ============================================================================
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(2) << 20;  // 2 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

__global__ void noalloc_write_job(FieldJob* dst, FieldJob job) { *dst = job; }

template <class T>
__global__ void noalloc_stage_in(const double* in, cpx<T>* dst, int n, int space) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int ix = q % n, iy = q / n;
  const bool unk = space == 2 ? (ix > 0 && iy > 0 && ix < n - 1 && iy < n - 1) : ((ix | iy) != 0);
  dst[q] = unk ? mkc<T>(T(in[2 * q]), T(in[2 * q + 1])) : czero<T>();
}

template <class T>
__global__ void noalloc_stage_out(const cpx<T>* src, double* out, int len) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  out[2 * q] = (double)src[q].x;
  out[2 * q + 1] = (double)src[q].y;
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <class T>
pint_status mg_noalloc_T(pint_ctx* c, Engine<T>& e, int which, int j, const double* in, double* out) {
  const Slots& s = c->s;
  const int J = c->J;
  const int space = which == 3 ? 1 : 2;
  int op;
  if (which == 0) {
    if (c->oseen) return c->fail(PINT_ERR_ARG, "W_j exists for Stokes problems only");
    op = j;
  } else if (which == 1 || which == 2) {
    if (!c->oseen) return c->fail(PINT_ERR_ARG, "Q_j exists for Oseen problems only");
    op = which == 1 ? j : J + j;
  } else {
    op = 2 * J;
  }
  const MGLayout& lay = space == 2 ? c->lay2 : c->lay1;
  const int n = space == 2 ? s.n2 : s.n1;
  const size_t field = (size_t)n * n * sizeof(cpx<T>);
  const size_t need = align256(sizeof(FieldJob)) + 2 * align256(field) + align256((size_t)lay.per_job * sizeof(cpx<T>));
  if (need > NOALLOC_SCRATCH_BYTES)
    return c->fail(PINT_ERR_ARG, "pint_mg_apply_noalloc: this field needs " + std::to_string(need) +
                                     " bytes of scratch, more than the fixed " +
                                     std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes");
  void* base = nullptr;
  if (!c->cu(noalloc_scratch(&base), "pint_mg_apply_noalloc scratch set-up")) return PINT_ERR_CUDA;
  unsigned char* p = static_cast<unsigned char*>(base);
  FieldJob* job = reinterpret_cast<FieldJob*>(p);
  p += align256(sizeof(FieldJob));
  cpx<T>* bfield = reinterpret_cast<cpx<T>*>(p);
  p += align256(field);
  cpx<T>* xfield = reinterpret_cast<cpx<T>*>(p);
  p += align256(field);
  cpx<T>* ws = reinterpret_cast<cpx<T>*>(p);

  FieldJob one{};
  one.nf = 1;
  one.op = op;
  noalloc_write_job<<<1, 1, 0, c->st>>>(job, one);
  noalloc_stage_in<T><<<(n * n + 255) / 256, 256, 0, c->st>>>(in, bfield, n, space);
  MGLaunch<T> L{};
  L.tabs = e.tabs;
  L.t64 = c->t64;
  for (int l = 0; l < PINT_MAXLEV; ++l) L.n2d[l] = e.n2d[l];
  L.fields_per_job = 1;
  L.cw = c->oseen && space == 2;
  L.lay = lay;
  L.ops = c->d_ops;
  L.coarse_inv = c->d_cinv;
  L.jobs = job;
  L.njobs = 1;
  L.xbase = xfield;
  L.bbase = bfield;
  L.ws = ws;
  L.active = nullptr;
  L.cycles = c->p.mg_cycles;
  L.pre = c->p.mg_pre;
  L.post = c->p.mg_post;
  L.omega = c->oseen && space == 2 ? c->omega_conv : c->p.sor_omega;
  L.space = space;
  L.conv = (which == 1 || which == 2) ? c->conv : false;
  L.no_tune = true;  // the tuner's bookkeeping allocates on the first launch of a shape
  launch_mg<T>(L, c->st);
  noalloc_stage_out<T><<<(n * n + 255) / 256, 256, 0, c->st>>>(xfield, out, n * n);
  return c->launched("pint_mg_apply_noalloc") ? PINT_OK : PINT_ERR_CUDA;
}

}  // namespace

extern "C" pint_status pint_mg_apply_noalloc(pint_handle h, int which, int j, const double* in, double* out) {
  if (!h || !in || !out) return g_err = "null argument", PINT_ERR_ARG;
  if (which < 0 || which > 3) return h->fail(PINT_ERR_ARG, "which must be a multigrid operator (0..3)");
  if (j < 0 || j >= h->J) return h->fail(PINT_ERR_ARG, "frequency index out of range");
  return h->fp32 ? mg_noalloc_T<float>(h, h->e32, which, j, in, out)
                 : mg_noalloc_T<double>(h, h->e64, which, j, in, out);
}

// ============================================================================
// Shared frequency solves for the serving loop (serve.cpp).
//
// Requests that share the grid, the domain, the wind, nu, the precision and
// the inner-solver settings form a group; their handles are members (role
// 1): each keeps its own outer FGMRES, KKT matvec and time DFT, while the
// frequency solves of all members that need a preconditioner apply at about
// the same time run as ONE batch in the group's shared context (role 2):
// every multigrid, Chebyshev, block-matvec and Gram-Schmidt launch covers the
// frequencies of all of them, each frequency with the constants of its own
// problem (tau, beta, n_t).  The frequencies are independent (Sec. 3.1), so a
// member's result does not depend on the other members of its batch.
// ============================================================================
#include <condition_variable>
#include <map>

#include "batch.h"

struct BatchMember {
  pint_ctx* c;
  void* R;
  void* Y;
  int* its;
  bool done;
  pint_status rc;
};

struct BatchGroup {
  pint_batcher_s* owner = nullptr;
  pint_params tmpl{};
  pint_ctx* b = nullptr;  // shared frequency-domain context (role 2), or null
  cudaStream_t st = nullptr;
  std::vector<BatchMember*> pending;
  bool running = false;
  int members = 0, in_solve = 0;
};

struct pint_batcher_s {
  std::mutex mu;
  std::condition_variable cv;
  std::map<std::string, BatchGroup*> groups;
  double window_ms = 3.0;  // how long a batch waits for members still in their outer step
  pint_group_stats stats{};
  // profile of the shared contexts (summed over batches; class APPLY = whole batches)
  std::mutex pmu;
  unsigned prof_mask = 0;
  pint_profile prof{};
};

namespace {

std::string group_key(const pint_params& p) {
  char k[512];
  snprintf(k, sizeof k, "%d|%d|%.17g|%.17g|%d|%.17g|%d|%.17g|%d|%d|%d|%d|%d|%d|%d|%.17g|%.17g|%.17g|%d", p.kind,
           p.level, p.x0, p.x1, p.wind, p.nu, p.prec, p.inner_tol, p.inner_maxit, p.fixed_inner_its, p.mg_cycles,
           p.mg_pre, p.mg_post, p.cheb_steps, p.uzawa_steps, p.uzawa_mu, p.sor_omega, p.sor_omega_conv, p.linear);
  return k;
}

pint_status make_ctx(const pint_params& p, int role, int cap, void* stream, pint_ctx** out) {
  pint_ctx* c = new (std::nothrow) pint_ctx();
  if (!c) return PINT_ERR_OOM;
  c->p = p;
  c->role = role;
  c->role_cap = cap;
  c->st = static_cast<cudaStream_t>(stream);
  const pint_status s = build(c);
  if (s != PINT_OK) {
    g_err = c->err;
    free_ctx(c);
    return s;
  }
  *out = c;
  return PINT_OK;
}

// One batch: the frequencies of every member, solved in the group's shared
// context (grown when the batch needs more frequencies than it holds).
pint_status run_batch(BatchGroup* g, std::vector<BatchMember*>& batch) {
  int jtot = 0;
  for (BatchMember* m : batch) jtot += m->c->J;
  if (!g->b || g->b->role_cap < jtot) {
    if (g->b) {
      free_ctx(g->b);
      g->b = nullptr;
    }
    const pint_status rc = make_ctx(g->tmpl, 2, jtot, g->st, &g->b);
    if (rc != PINT_OK) return rc;
  }
  pint_ctx* b = g->b;
  std::vector<FreqDesc> fd;
  fd.reserve(jtot);
  for (BatchMember* m : batch)
    for (int j = 0; j < m->c->J; ++j) fd.push_back(FreqDesc{m->c->p.tau, m->c->p.beta, m->c->K, j});
  pint_status rc = fill_freq_tables(b, fd);
  if (rc != PINT_OK) return rc;
  const size_t cb = b->fp32 ? sizeof(cpx<float>) : sizeof(cpx<double>);
  const size_t nb = (size_t)b->s.nblk;
  char* Rb = static_cast<char*>(b->fp32 ? (void*)b->e32.R : (void*)b->e64.R);
  char* Yb = static_cast<char*>(b->fp32 ? (void*)b->e32.Y : (void*)b->e64.Y);
  size_t off = 0;
  for (BatchMember* m : batch) {
    const size_t bytes = (size_t)m->c->J * nb * cb;
    if (!b->cu(cudaMemcpyAsync(Rb + off, m->R, bytes, cudaMemcpyDeviceToDevice, b->st), "batch input"))
      return PINT_ERR_CUDA;
    off += bytes;
  }
  std::vector<int> its(jtot, 0);
  {
    std::lock_guard<std::mutex> pk(g->owner->pmu);
    b->prof_mask = g->owner->prof_mask;
  }
  {
    PROF(b, PINT_PROF_APPLY, 0);
    if (b->fp32)
      b->e32.freq_solve(b->e32.R, b->e32.Y, its.data());
    else
      b->e64.freq_solve(b->e64.R, b->e64.Y, its.data());
  }
  off = 0;
  int j0 = 0;
  for (BatchMember* m : batch) {
    const size_t bytes = (size_t)m->c->J * nb * cb;
    if (!b->cu(cudaMemcpyAsync(m->Y, Yb + off, bytes, cudaMemcpyDeviceToDevice, b->st), "batch output"))
      return PINT_ERR_CUDA;
    if (m->its) std::copy(its.begin() + j0, its.begin() + j0 + m->c->J, m->its);
    off += bytes;
    j0 += m->c->J;
  }
  if (!b->launched("shared frequency solve") || !b->cu(cudaStreamSynchronize(b->st), "shared frequency solve"))
    return PINT_ERR_CUDA;
  ++b->prof_syncs;
  if (b->st_aux) cudaStreamSynchronize(b->st_aux);
  b->drain();
  {
    // fold this batch's counters into the group's profile
    std::lock_guard<std::mutex> pk(g->owner->pmu);
    pint_profile& P = g->owner->prof;
    for (int i = 0; i < PINT_PROF_CLASSES; ++i) {
      P.launches[i] += b->prof_launch[i];
      P.timed[i] += b->prof_timed[i];
      P.ms[i] += b->prof_ms[i];
      P.bytes[i] += b->prof_bytes[i];
      b->prof_launch[i] = b->prof_timed[i] = 0;
      b->prof_ms[i] = b->prof_bytes[i] = 0.0;
    }
    P.host_syncs += b->prof_syncs;
    b->prof_syncs = 0;
  }
  return PINT_OK;
}

}  // namespace

pint_status shared_freq_solve(pint_ctx* c, void* R, void* Y, int* its_host) {
  BatchGroup* g = c->group;
  pint_batcher_s* B = g->owner;
  if (!c->cu(cudaStreamSynchronize(c->st), "member DFT")) return PINT_ERR_CUDA;
  BatchMember me{c, R, Y, its_host, false, PINT_OK};
  std::unique_lock<std::mutex> lk(B->mu);
  g->pending.push_back(&me);
  B->cv.notify_all();
  while (!me.done) {
    if (!g->running && !g->pending.empty()) {
      // this thread runs the next batch (one batch of a group at a time):
      // first wait (bounded) for the members that are still in their outer step
      g->running = true;
      const auto deadline = std::chrono::steady_clock::now() +
                            std::chrono::microseconds((long long)(B->window_ms * 1000.0));
      while ((int)g->pending.size() < g->in_solve && std::chrono::steady_clock::now() < deadline)
        B->cv.wait_until(lk, deadline);
      std::vector<BatchMember*> batch;
      batch.swap(g->pending);
      lk.unlock();
      const pint_status rc = batch.empty() ? PINT_OK : run_batch(g, batch);
      lk.lock();
      int nf = 0;
      for (BatchMember* m : batch) {
        m->rc = rc;
        m->done = true;
        nf += m->c->J;
      }
      B->stats.batches++;
      B->stats.member_solves += (long long)batch.size();
      B->stats.frequencies += nf;
      B->stats.max_members = std::max(B->stats.max_members, (int)batch.size());
      if (rc != PINT_OK) c->err = g_err = "shared frequency solve failed: " + g_err;
      g->running = false;
      B->cv.notify_all();
    } else {
      B->cv.wait(lk);
    }
  }
  return me.rc;
}

pint_batcher_s* batcher_create() { return new pint_batcher_s(); }

void batcher_destroy(pint_batcher_s* B) {
  if (!B) return;
  for (auto& kv : B->groups) {
    if (kv.second->b) free_ctx(kv.second->b);
    if (kv.second->st) cudaStreamDestroy(kv.second->st);
    delete kv.second;
  }
  delete B;
}

pint_status member_create(pint_batcher_s* B, const pint_params* p, void* stream, pint_handle* out) {
  std::string why;
  if (!valid_params(p, why)) return g_err = why, PINT_ERR_ARG;
  if (p->wind == PINT_WIND_NODAL) return g_err = "shared solves take the built-in winds only", PINT_ERR_ARG;
  pint_ctx* c = nullptr;
  const pint_status rc = make_ctx(*p, 1, 0, stream, &c);
  if (rc != PINT_OK) return rc;
  std::lock_guard<std::mutex> lk(B->mu);
  BatchGroup*& g = B->groups[group_key(*p)];
  if (!g) {
    g = new BatchGroup();
    g->owner = B;
    g->tmpl = *p;
    cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking);
  }
  g->members++;
  c->group = g;
  *out = c;
  return PINT_OK;
}

void member_destroy(pint_handle h) {
  if (!h) return;
  BatchGroup* g = h->group;
  if (g) {
    std::lock_guard<std::mutex> lk(g->owner->mu);
    if (--g->members == 0 && g->b && !g->running) {
      free_ctx(g->b);  // the group's memory goes back with its last member
      g->b = nullptr;
    }
  }
  free_ctx(h);
}

static void member_solve_begin(pint_handle h) {
  std::lock_guard<std::mutex> lk(h->group->owner->mu);
  h->group->in_solve++;
  h->in_solve = true;
}

static void member_solve_end(pint_handle h) {
  std::lock_guard<std::mutex> lk(h->group->owner->mu);
  h->group->in_solve--;
  h->in_solve = false;
  h->group->owner->cv.notify_all();
}

void batcher_get_stats(pint_batcher_s* B, pint_group_stats* out) {
  std::lock_guard<std::mutex> lk(B->mu);
  *out = B->stats;
}

// Device bytes a member holds, and what one frequency adds to its group's
// shared context (upper estimates, host arithmetic only).
void shared_estimates(const pint_params* p, size_t* member_bytes, size_t* per_freq_bytes) {
  const long long N = 1LL << p->level, K = p->n_t, J = K / 2 + 1;
  const long long ns = (2 * N + 1) * (2 * N + 1), nq = (N + 1) * (N + 1), nblk = 4 * ns + 2 * nq;
  const bool fp32 = p->prec == PINT_PREC_FP32, oseen = p->kind == PINT_OSEEN;
  const long long cs = fp32 ? 8 : 16;
  const long long m = p->outer_restart;
  const long long m_in = p->fixed_inner_its > 0 ? p->fixed_inner_its : p->inner_maxit;
  long long mb = (2 * m + 4) * K * nblk * 8 + J * nblk * 16 + 2 * J * nblk * cs;
  *member_bytes = (size_t)(mb + mb / 20 + (64LL << 20));
  long long f = 3 * nblk * cs;
  if (!p->linear) f += (2 * m_in + 1) * nblk * cs + (m_in + 1) * m_in * 16 * 2;
  const MGLayout l2 = make_layout(p->level, (int)N, 2), l1 = make_layout(p->level, (int)N, 1);
  f += std::max((oseen ? 2 : 4) * l2.per_job, 2 * l1.per_job) * cs;
  if (!oseen) f += 2 * l1.per_job * cs;
  f += std::max((long long)(oseen ? 2 : 0) * 2 * ns, 2LL * 2 * nq) * cs;
  *per_freq_bytes = (size_t)(f + f / 20);
}

extern "C" {

pint_status pint_group_create(pint_group* out) {
  if (!out) return g_err = "null argument", PINT_ERR_ARG;
  *out = batcher_create();
  return PINT_OK;
}

pint_status pint_create_in_group(pint_group g, const pint_params* p, void* stream, pint_handle* out) {
  if (!g || !p || !out) return g_err = "null argument", PINT_ERR_ARG;
  *out = nullptr;
  return member_create(g, p, stream, out);
}

pint_status pint_group_get_stats(pint_group g, pint_group_stats* out) {
  if (!g || !out) return g_err = "null argument", PINT_ERR_ARG;
  batcher_get_stats(g, out);
  return PINT_OK;
}

pint_status pint_group_profile_enable(pint_group g, unsigned mask) {
  if (!g) return g_err = "null group", PINT_ERR_ARG;
  std::lock_guard<std::mutex> pk(g->pmu);
  g->prof_mask = mask;
  g->prof = pint_profile{};
  return PINT_OK;
}

pint_status pint_group_profile_read(pint_group g, pint_profile* out) {
  if (!g || !out) return g_err = "null argument", PINT_ERR_ARG;
  std::lock_guard<std::mutex> pk(g->pmu);
  *out = g->prof;
  return PINT_OK;
}

pint_status pint_group_destroy(pint_group g) {
  batcher_destroy(g);
  return PINT_OK;
}

}  // extern "C"
