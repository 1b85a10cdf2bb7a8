// Internal declarations of libmrcm: host plan, workspace layout, handle, kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/mrcm.h"

#include <cuda_runtime_api.h>

namespace mrcm {

// ------------------------------------------------------------------------------------------
// Host plan: partition and coupling-system numbering (MRCM-OS step 1), integer only.
// ------------------------------------------------------------------------------------------
// One front of the nested-dissection multifrontal factorisation of G: the pivot unknowns P (the
// interfaces on the separator of its rectangle of subdomains, or every interface inside a leaf
// rectangle) and the update unknowns U (the interfaces on the rectangle's boundary), P first.  The
// dense front F = [F11 F12; F21 F22] (row-major, f = np + nu) is overwritten by F11^-1,
// D = F11^-1 F12 and S = F22 - F21 D; B = F21 F11^-1 (nu x np) follows F.
struct MfFront {
  long long fo;   // offset (doubles) of F in the front buffer
  int np, nu;
  int io;         // first of its np + nu unknowns in the index list
  int vo;         // offset (doubles) of its solve vectors [v_P, w_U]
  int ao, na;     // its assembly pairs
  int nch;        // children (0..2)
  int ch[2];      // child front ids
  int mo[2];      // offsets of the children's maps
  int par;        // parent front id (-1 at the root)
};
constexpr int MF_LEAF = 16;       // leaf rectangles of at most this many subdomains
constexpr int MF_MAX_NP = 128;    // largest pivot block (its inverse is formed in shared memory)
constexpr int MF_TILE = 32;       // tile of the D, B and S products

struct Plan {
  int dim = 2;
  int n[3] = {1, 1, 1};
  int sub[3] = {1, 1, 1};
  int m[3] = {1, 1, 1};     // subdomains per axis
  int l = 0;
  int S = 0;                // subdomains
  int E = 0;                // interfaces
  int E2 = 0;               // Robin sides = 2E
  int nq = 1;               // polynomial functions per Robin side (1 + interface degree)
  int NC = 0;               // coupling unknowns = 2E nq
  std::vector<int> box;     // [S][6] lo[3] hi[3]
  std::vector<int> obox;    // [S][6] oversampled box clipped to the grid
  std::vector<int> mask;    // [S] Robin side bits
  std::vector<int> N;       // [S]
  std::vector<int> off;     // [S] first coarse unknown
  std::vector<int> rank;    // [S][6] rank among the Robin sides, -1 if not Robin
  std::vector<int> iface;   // [E][3] axis, lower s, upper s
  // coupling rows in the banded "home" order: the flux row of interface e sits at the unknown of
  // the lower subdomain's +axis side, the pressure row at the upper subdomain's -axis side
  std::vector<int> row_home;   // [2E] canonical row -> banded row
  int kl = 0, ku = 0;          // band widths of G in the banded order
  // nested-dissection multifrontal factorisation of G (2-D coupling systems above
  // COARSE_DENSE_MAX unknowns; mf is set when every front fits the kernels of k_mf.cu)
  bool mf = false;
  std::vector<MfFront> mf_front;   // postorder (children before parents)
  std::vector<int> mf_order;       // front ids grouped by level (leaves are level 0)
  std::vector<int> mf_level;       // [levels + 1] starts of the levels in mf_order
  std::vector<int> mf_idx;         // unknowns of each front, P then U
  std::vector<int> mf_asm;         // (dst, src) pairs: front-local offset, band offset of G
  std::vector<int> mf_map;         // child U position -> parent front position
  std::vector<int> mf_task;        // (front, kind, r0, c0) tile tasks
  std::vector<int> mf_task_b;      // [levels + 1] starts of each level's D / B tasks
  std::vector<int> mf_task_c;      // [levels + 1] starts of each level's Schur-complement tasks
  size_t mf_fbuf = 0;              // doubles of all fronts (F and B)
  size_t mf_vbuf = 0;              // doubles of the solve vectors
  int mf_max_np = 0, mf_max_f = 0;
  int mf_mcap = 0;                 // front rows staged by the solve (doubles, padded rows): the largest B or
                                   // [F11^-1 D], capped at 24576 (192 KB)
};

// Returns an empty string on success, else the reason the input is invalid.
std::string make_plan(const mrcm_problem& p, const mrcm_params& q, Plan& plan);
std::vector<int32_t> export_plan(const Plan& plan);

// ------------------------------------------------------------------------------------------
// Workspace layout (byte offsets, 256-byte aligned).
// ------------------------------------------------------------------------------------------
struct Layout {
  size_t K, Ky, Tx, Ty, b, f, bcv;        // problem data (Ky: y component of K; bcv: 4 side arrays)
  size_t Linv_loc, Linv_ohat_r, Linv_ohat_d;   // line-block inverse factors
  size_t phi, psi, mom, psi0, z0, mom0;   // informed spaces, basis, side moments, apply scratch
  size_t coef_o, coef_l;                  // FP64 line coefficients of the Robin boxes (FP32 local solves)
  size_t G, ipiv, gc;                     // coupling band LU, pivots, rhs / solution
  size_t rdiag;                           // reciprocals of the diagonal of U
  size_t Ginv;                            // dense inverse of G (when 2E <= COARSE_DENSE_MAX)
  size_t gtr;                             // Robin coefficients of the Gamma faces, k_local.cu
  size_t rto, rtl;                        // t_R of the Robin box faces of the oversampled / subdomain boxes
  size_t gbML, gbMU, gbX, gbY, gbF, gbC;  // blocked substitution (above COARSE_DENSE_MAX), k_coarse.cu
  size_t mf_fr, mf_ord, mf_lvl, mf_idx, mf_asm, mf_map, mf_task;   // multifrontal tables, k_mf.cu
  size_t mf_F, mf_V, mf_scr, mf_done;     // fronts, solve vectors, scratch words, completion flags
  size_t rho, zt;                         // FP32 staged right-hand sides (k_stage32), apply output scratch
  size_t V, Z, w, Hs, red, flags, tmpv;   // Krylov basis and scratch
  size_t tab;                             // device copies of the plan tables
  size_t apart, atot, aT;                 // Arnoldi partial sums, totals, (I + R)^-1
  size_t total;
  // sizes
  int wl, wo;             // line width of the Omega and hat-Omega boxes
  int hl, ho;             // line count (box height)
  int LSl, LSo;           // packed line-block stride (elements) for each box kind
  int ldab;               // leading dimension of the coupling band
  int smax;               // max(sub0, sub1)
  int m;                  // restart length
  int nred;               // reduction partial count
  size_t elt;             // bytes per local-factor element
};
Layout make_layout(const Plan& plan, const mrcm_params& q);

// ------------------------------------------------------------------------------------------
// Device-side geometry passed by value to kernels (2-D).
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__
#define MRCM_HD __host__ __device__
#else
#define MRCM_HD
#endif
// Elements per box of a line-block factor array: h packed line blocks of LS elements, then the
// h x w line couplings (coupling of each cell to the line below), padded to a 16-byte multiple.
MRCM_HD inline size_t box_stride(int w, int h, int LS) {
  return (size_t)h * LS + (((size_t)h * w + 3) & ~(size_t)3);
}

struct Geo {
  int nx, ny;
  int sx, sy;              // subdomain size
  int mx, my;              // subdomain counts
  int l;                   // oversampling
  int smax;
  int nq;                  // functions per Robin side
  double hx, hy, hz;
  double alpha;
  const double* K;         // scalar permeability, or the x component of a diagonal tensor
  const double* Ky;        // the y component (equal to K for a scalar field)
  const double* Tx;        // ny x (nx+1)
  const double* Ty;        // (ny+1) x nx
  const double* rto = nullptr;   // [S][4 sides][rlo] t_R of the Robin faces of the oversampled boxes (0 elsewhere)
  const double* rtl = nullptr;   // [S][4 sides][rll] the same for the subdomain boxes; both written once per set-up
  int rlo = 0, rll = 0;          // (k_robin_tab) and read by the factorisations and the informed solves
  double* gtr = nullptr;   // [S][4 sides][smax] x (t_R, beta, T_f, |f| / tau) of the Gamma faces: written once per
                           // set-up (k_gamma_coef), read by the informed, basis and particular solves
};

// ------------------------------------------------------------------------------------------
// Device scratch for deterministic reductions: per-block partials + a completion counter.
// ------------------------------------------------------------------------------------------
constexpr int RED_BLOCKS = 608;   // 152 SMs x 4
constexpr int RED_THREADS = 256;
constexpr int ARNOLDI_MAX_BLOCKS = 1024;
// reduction scratch (doubles): [0, 4096) classic partials, [4096, 8192) Arnoldi partials,
// then unsigned counters: [0] classic ticket, [1] barrier arrivals, [2] barrier generation
constexpr size_t RED_DOUBLES = 8192;
constexpr int COARSE_DENSE_MAX = 4096;   // 2E up to this size: explicit G^-1, one product per apply
constexpr int GBB_NB = 512;              // above it: substitution steps per block of the blocked solve

// flag word bits (device status)
enum : int { FLAG_SINGULAR_LOCAL = 1, FLAG_SINGULAR_COARSE = 2, FLAG_NONFINITE = 4, FLAG_TIMEOUT = 8,
             FLAG_NOPIV_REJECTED = 16 };   // the no-pivot coupling LU met a zero pivot or large growth

}  // namespace mrcm

// The handle.
struct mrcm_ctx {
  mrcm::Plan plan;
  mrcm::Layout lay;
  mrcm_params prm;
  int dim;
  int n[3];
  double h[3];
  int bc_kind[6];
  int has_bc[6];
  int has_f;
  bool iso = true;    // K is a scalar field (Ky mirrors it)
  int device = -1;    // the device current at mrcm_setup (the workspace's device)
  char* ws;           // workspace base (device)
  size_t ws_bytes;
  bool factored = false;
  bool coarse_pivoted = false;   // the last factorisation of G fell back to partial pivoting
  bool coarse_mf = false;        // G factored by the multifrontal LU (k_mf.cu)
  std::string err;
  int coarse_n;       // 2E
  std::vector<int> tab_host;  // plan tables uploaded to the device
  bool keep_z0 = false;       // keep the last multiscale solution for debug reads
  const volatile int* cancel = nullptr;  // set by the request server; checked once per GMRES step
  // phase profiler
  bool prof = false;
  uint32_t prof_mask = ~0u;     // phases recorded while prof is set
  int prof_every = 1;           // record every prof_every-th occurrence of a phase
  long long ph_seen[MRCM_PHASES] = {0};   // occurrences of each phase since the last selection
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_phase;   // phase of each recorded (start, stop) pair, in pool order
  size_t ev_used = 0;          // pairs recorded since the last read
  double ph_ms[MRCM_PHASES] = {0};
  long long ph_launch[MRCM_PHASES] = {0};
  // GMRES step read-back: pinned slots so that step j's residual estimate is read while step j+1
  // runs (created on the first solve)
  struct StepReadback {
    double out[4];
    int flags;
    int pad;
  };
  StepReadback* rb = nullptr;
  cudaEvent_t rb_ev[2] = {nullptr, nullptr};
  // second stream for set-up work that overlaps (the Schwarz factors), with its fork / join events
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr, omega_ev = nullptr;
  ~mrcm_ctx() {
    if (side) cudaStreamDestroy(side);
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (join_ev) cudaEventDestroy(join_ev);
    if (omega_ev) cudaEventDestroy(omega_ev);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : rb_ev)
      if (e) cudaEventDestroy(e);
    if (rb) cudaFreeHost(rb);
  }
};

namespace mrcm {
void count_launch(int kernels);
// message returned by mrcm_last_error(NULL) on the calling thread
void set_thread_error(const std::string& msg);
// kernel launchers (k_*.cu)
cudaError_t launch_assemble(const Geo& g, const int* bc_kind, const double* const* bcv, const double* f,
                            double* Tx, double* Ty, double* b, cudaStream_t st);
cudaError_t launch_matvec(const Geo& g, const double* v, double* w, cudaStream_t st);
cudaError_t launch_residual(const Geo& g, const double* r, const double* z, double* rho, cudaStream_t st);
// FP64 FMA throughput probe (k_grid.cu): blocks x threads x iters x 32 FMA
cudaError_t launch_dfma_probe(double* sink, int blocks, int threads, int iters, cudaStream_t st);
cudaError_t launch_fluxes(const Geo& g, const int* bc_kind, const double* const* bcv, const double* p,
                          double* ux, double* uy, cudaStream_t st);

// local factor / solve (k_local.cu)
enum BoxKind : int { BOX_OMEGA_ROBIN = 0, BOX_OHAT_ROBIN = 1, BOX_OHAT_DIRICHLET = 2 };
// coef (optional): the box kind's FP64 line coefficients [S][h][w][d, o, e], written on the way
cudaError_t launch_factor(const Geo& g, int kind, int w, int hgt, int LS, void* Linv, bool fp32, int* flags,
                          cudaStream_t st, double* coef = nullptr);
// each cell's FP64 line coefficients [S][h][w][diagonal, x coupling, y coupling] of the boxes of
// one kind; given to the FP32 informed and basis solves (coef), they refine once against them
cudaError_t launch_line_coef(const Geo& g, int kind, double* coef, cudaStream_t st);
// the Robin coefficients of every Gamma face into g.gtr (after the transmissibilities)
cudaError_t launch_gamma_coef(const Geo& g, cudaStream_t st);
// t_R of the Robin faces of every oversampled (ohat) or subdomain box into its table, g.rto or g.rtl
// (once per set-up, before the factorisation of that kind; needs K only)
cudaError_t launch_robin_tab(const Geo& g, bool ohat, double* out, cudaStream_t st);
cudaError_t launch_informed(const Geo& g, const void* Linv, int LS, bool fp32, double* phi, int q, int* flags, cudaStream_t st,
                            const double* coef = nullptr);
cudaError_t launch_basis(const Geo& g, const void* Linv, int LS, bool fp32, const double* phi, int q, double* psi,
                         double* mom, int* flags, cudaStream_t st, const double* coef = nullptr);
// FP32 right-hand sides formed once on the grid for the FP32 particular solves (z == nullptr: r) and
// additive sweeps (the residual r - A z in FP64, rounded once): n floats into out
cudaError_t launch_stage32(const Geo& g, const double* r, const double* z, float* out, cudaStream_t st);
// in32 (FP32 solves, optional): the right-hand side staged by launch_stage32 for this launch (the
// particular solve's r, or the additive sweep's residual for the same zin); null: formed per box
cudaError_t launch_particular(const Geo& g, const void* Linv, int LS, bool fp32, const double* r, double* psi0,
                              double* mom0, int* flags, cudaStream_t st, const float* in32 = nullptr);
cudaError_t launch_schwarz(const Geo& g, const void* Linv, int LS, bool fp32, const double* r, const double* zin,
                           double* zout, int* flags, int colour, cudaStream_t st, const float* in32 = nullptr);
cudaError_t launch_reconstruct(const Geo& g, const double* psi0, const double* psi, const int* coff,
                               const double* c, double* z, cudaStream_t st);
size_t factor_smem_bytes(int w, bool fp32, int nch);

// coupling system (k_coarse.cu)
struct CoarseDev {
  int n;            // 2E nq
  int nq;           // functions per Robin side
  int kl, ku, ldab;
  double* ab;       // band LU storage, column-major, ldab x n
  int* ipiv;
  double* rdiag;    // 1 / U(j, j), written by the factorisation
  // blocked substitution (2E nq > COARSE_DENSE_MAX): nbk blocks of GBB_NB steps; per block the dense
  // transform of its L steps (window GBB_NB + kl) and of its U steps (window GBB_NB + kl + ku),
  // column-major; padded vectors (kl + ku leading and kl trailing zeros); fresh-input products
  // [nbk][GBB_NB + kl + ku]; carries entering each block [nbk][kl + ku]
  int nbk;
  double *ML, *MU, *X, *Y, *F, *C;
  double* g;        // rhs / solution (banded row order in, canonical unknowns out)
  const int* iface; // [E][3]
  const int* home;  // [2E] canonical row -> banded row
  const int* off;   // [S]
  const int* rank;  // [S][6]
};
cudaError_t launch_coarse_assemble(const CoarseDev& c, const double* mom, int E, cudaStream_t st);
// variant: see k_coarse.cu (-1: the first that runs); coarse_factor_variants lists those that run
cudaError_t launch_coarse_factor(const CoarseDev& c, int* flags, cudaStream_t st, int variant = -1);
constexpr int COARSE_FACTOR_MAX_VARIANTS = 8;
int coarse_factor_variants(const CoarseDev& c, int* v);   // v: COARSE_FACTOR_MAX_VARIANTS entries
cudaError_t launch_coarse_rhs(const CoarseDev& c, const double* mom0, int E, cudaStream_t st);
// per apply without an explicit inverse: right-hand side from mom0, then the band solve
cudaError_t launch_coarse_solve(const CoarseDev& c, const double* mom0, int E, cudaStream_t st);
cudaError_t launch_coarse_invert(const CoarseDev& c, double* Ginv, cudaStream_t st);
// Band LU of G without row interchanges (identity ipiv), blocked over the whole GPU in one
// cooperative launch; sets FLAG_NOPIV_REJECTED when a pivot is zero or not finite or an element
// grows past NOPIV_MAX_GROWTH times the largest entry of G (the caller then factors with pivoting).
// scratch: 8 words of device memory (barrier and statistics), zeroed by the launcher.
constexpr double NOPIV_MAX_GROWTH = 1e6;
cudaError_t launch_coarse_factor_nopiv(const CoarseDev& c, int* flags, unsigned* scratch, cudaStream_t st);
// set-up of the blocked substitution (2E nq > COARSE_DENSE_MAX), after the factorisation
cudaError_t launch_coarse_blocks(const CoarseDev& c, cudaStream_t st);
cudaError_t launch_coarse_apply(const CoarseDev& c, const double* Ginv, const double* mom0, int E, cudaStream_t st);

// Multifrontal factorisation of G (k_mf.cu): device copies of the plan's tables and buffers.
struct MfDev {
  const MfFront* fr;
  const int* order;
  const int* lvl;       // [levels + 1]
  const int* idx;
  const int2* asmv;
  const int* map;
  const int4* task;
  double* F;
  double* V;
  unsigned* scr;        // [2, 6) two 8-byte maxima (|G| entries, |S| entries); [8] solve epoch,
                        // [9] CTAs finished in the current solve
  unsigned* done;       // [2 nfront] forward / backward completion epochs of each front
  int levels;
  int nfront;
  int max_f;            // largest front (np + nu)
  int mcap;             // doubles of front rows the solve stages in shared memory
};
// Set-up: fronts level by level (assembly from the band copy of G and F11^-1, then the D and B
// tiles, then the Schur-complement tiles) and a final growth check that sets FLAG_NOPIV_REJECTED
// when a pivot is zero or not finite or |S| grows past NOPIV_MAX_GROWTH max |G| (the caller then
// falls back to the pivoted band LU).
cudaError_t launch_mf_factor(const MfDev& m, const Plan& P, const double* ab, int* flags, cudaStream_t st);
// Per apply: right-hand side from mom0 (through c), then one cooperative launch: forward through
// the levels, backward down them, each front waiting on its children's (parent's) completion
// flags; the solution replaces c.g.
cudaError_t launch_mf_solve(const MfDev& m, const CoarseDev& c, const double* mom0, int E, int* flags,
                            cudaStream_t st);
cudaError_t launch_arnoldi(const Geo& g, const double* z, double* V, int j, size_t n, double* H, int ldh, double* cs,
                           double* sn, double* gv, double* out, double* wbuf, double* part, double* tot, double* Tm,
                           unsigned* bar, int* flags, cudaStream_t st);

// Krylov helpers (k_krylov.cu)
cudaError_t launch_norm2(const double* x, size_t n, double* partials, unsigned* counter, double* out,
                         cudaStream_t st);
cudaError_t launch_scale(const double* x, const double* denom, size_t n, double* y, cudaStream_t st);
cudaError_t launch_matvec_dot(const Geo& g, const double* z, const double* v0, double* w, double* partials,
                              unsigned* counter, double* out2, cudaStream_t st);
cudaError_t launch_mgs_pass(const double* vprev, const double* hprev, const double* vnext, size_t n, double* w,
                            double* partials, unsigned* counter, double* hout, int want_norm, cudaStream_t st);
cudaError_t launch_givens(double* H, double* cs, double* sn, double* gv, int j, int ldh, double* hnorm0,
                          double* out, cudaStream_t st);
cudaError_t launch_update(double* p, const double* Z, size_t n, const double* H, const double* gv, int k, int ldh,
                          double* ybuf, cudaStream_t st);
cudaError_t launch_residual_norm(const Geo& g, const double* b, const double* p, double* r, double* partials,
                                 unsigned* counter, double* out, cudaStream_t st);
// Launch-shape autotuning (tune.cpp).  autotune() returns the index of the fastest of ncand
// variants of shape (kind, key) -- timing them on the stream with run(i), which must give the same
// result for every i and may be repeated -- or -1 for the caller's built-in choice (tuning off,
// the shape being timed by another thread, or a stream under capture).
int autotune(int kind, const int key[6], int ncand, cudaStream_t st, const std::function<cudaError_t(int)>& run,
             cudaError_t* err);
void autotune_mode(int mode);            // 0 off (built-in choices), 1 on, 2 forget the tuned shapes and turn on
std::vector<double> autotune_table();    // per tuned shape: kind, key[6], choice, ncand, best us
enum : int { TUNE_LOCAL_SOLVE = 0, TUNE_COARSE_FACTOR = 1 };

}  // namespace mrcm
