// sadi_internal.h -- launch wrappers shared by the translation units of the
// S-ADI library.  Not part of the public C ABI (include/sadi.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

namespace sadi {

// Sizes of one instance.  N interior points per direction; the FFT length
// Np = N' is the smallest power of two >= max(N, 8); the 2D convolution works
// on the 2Np x 2Np block-circulant embedding (P = 2Np >= 2N - 1); the
// Gohberg-Semencul solves work on the bordered Np x Np Toeplitz matrix with
// border rank r = Np - N.
struct Geom {
  int N, Np, logNp, P, logP, r;
  // row pitch (elements) of the context's N x N arrays (state, sweep scratch,
  // phi2, source, remainder pair): N for FP64, N rounded up to a multiple of
  // kPitchAlign for the FP32 forms (aligned rows for vector accesses)
  int ld;
};
constexpr int kPitchAlign = 32;

// Scalars of the right-hand side B^n (Sec. 3): tau, tau^2, g kind, n == 0.
// g kinds: 0 none, 1 -u^3, 2 -sin u, 3 gc1 u + gc3 u^3 + gcs sin u.
// eq 0: the wave equation (tau2 = tau^2); eq 1: the diffusion equation
// (tau2 = tau), B = tau (-kappa L_h u~ + g(u~) + f) - d with d = u^n - u^{n-1}
// and u~ = u^n + d/2 (d = 0 at n = 0).
struct RhsParams {
  int eq;
  double tau, tau2;
  int g;
  int first;
  const void* F;   // optional source field (T, N x N) or nullptr
  double fsc;      // its time factor cos(omega t_n + phase) for this step
  double gc1, gc3, gcs;   // coefficients of g kind 3
};

// ---- setup (FP64), setup_kernels.cu ----------------------------------------
cudaError_t launch_twiddles(double2* tw64, float2* tw32, int P, cudaStream_t st);
// per-stage FFT twiddle tables of the length-2^logL plan (fft_plan)
cudaError_t launch_stage_twiddles(double2* stw64, float2* stw32, int logL, cudaStream_t st);
cudaError_t launch_riesz1d(double* a, int n, double alpha, cudaStream_t st);
// 2D weights a_ij (0 <= i, j < N) by the trapezoid rule on grids M and 2M +
// one Richardson step.  Scratch is allocated and freed inside.
cudaError_t run_weights2d(double* a2d, const Geom& g, double alpha, int M, const double2* stw64,
                          cudaStream_t st);
// Symbol of the block-circulant embedding: lnat[(Np+1) x (Np+1)] (unscaled,
// natural order), and the bit-reversed conv tables lpb (scaled) in FP64/FP32.
cudaError_t run_lambda(const double* a2d, const Geom& g, const double2* stw64, const double2* tw64, double scale,
                       double* lnat,
                       double* lpb64, float* lpb32, cudaStream_t st);
// Gohberg-Semencul generator of H' = I + s T(a_0..a_{Np-1}): c' (Np), spectra
// lam_c, lam_s (bit-reversed, scaled) and border correction G (N x r).
// *status_host receives 0 on success, 1 if the Durbin recursion broke down.
cudaError_t run_generator(const double* a1, const Geom& g, double s, const double2* stw64, const double2* tw64,
                          double* cgen,
                          double2* lamc64, double2* lams64, float2* lamc32, float2* lams32, double* G64,
                          float* G32, int* status_host, cudaStream_t st);
// Element-wise conversions of a rows x cols array, source rows sld elements
// apart, destination rows dld apart (padding elements are not touched).
cudaError_t launch_convert_d2f(const double* src, float* dst, int rows, int cols, int sld, int dld, cudaStream_t st);
cudaError_t launch_convert_f2d(const float* src, double* dst, int rows, int cols, int sld, int dld, cudaStream_t st);
// double -> (hi, lo) float pair; (hi, lo) -> double hi + lo, or float hi + lo
cudaError_t launch_split_d2ff(const double* src, float* hi, float* lo, int rows, int cols, int sld, int dld,
                              cudaStream_t st);
cudaError_t launch_join_ff2d(const float* hi, const float* lo, double* dst, int rows, int cols, int sld, int dld,
                             cudaStream_t st);
cudaError_t launch_join_ff2f(const float* hi, const float* lo, float* dst, int rows, int cols, int sld, int dld,
                             cudaStream_t st);

// ---- per-step kernels, step_kernels.cu --------------------------------------
template <typename T>
struct StepTables {
  const void* stw;     // cx<T>[plan.total]  per-stage FFT twiddles
  const void* tw;      // cx<T>[P]
  const T* lpb;        // [(Np+1) * 2 * Np]
  const void* lam_s;   // cx<T>[Np]
  const void* lam_c;   // cx<T>[Np]
  const T* G;          // [N * r]
  const struct Conv3* c3 = nullptr;   // FP32, N' = 2048 .. 8192: three-pass column convolution
};

// One-time launcher state (kernel attributes, launch shapes) is per device:
// launchers keep it in arrays indexed by the current device.  Host threads
// driving different contexts may make a device's first launches at the same
// time, so a cached value is stored (release) only after what it vouches for
// (the kernel attributes) has been set, and loaded with acquire; 0 = not yet.
constexpr int kLauncherDevices = 64;
using LaunchCache = std::atomic<int>;
inline int device_slot() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kLauncherDevices) return -1;
  return d;
}

// ---- three-pass column convolution (FP32, N' = 2048 .. 8192), conv3.cu -----
// N' = R1 x 64; ZE / ZO hold the even / odd frequency halves between the
// passes (N' rows x CW = N' + 16 columns); Lt is the symbol re-laid for the
// middle pass; twM[k] = exp(-2 pi i k / N'); tw1a / tw1b are the twiddles of
// the 64-point and R1-point register transforms.
struct Conv3 {
  float2* ZE = nullptr;
  float2* ZO = nullptr;
  float* Lt = nullptr;
  float2* twM = nullptr;
  float2* tw1a = nullptr;
  float2* tw1b = nullptr;
  int CW = 0, R1 = 0, logR1 = 0;
};
bool conv3_supported(int logNp);   // FFT lengths its kernels serve (2048 .. 8192)
// allocate and fill the buffers and tables (once per context); lpb32 is the
// shared-memory engine's symbol table
cudaError_t conv3_setup(int Np, int logNp, const float* lpb32, Conv3* c, cudaStream_t st);
void conv3_free(Conv3* c);
// the convolution of every column of the FP32 spectrum S (N x N' float2) in
// place; tw is the float2 table exp(-2 pi i k / 2N')
cudaError_t launch_conv3(const Conv3& c, int N, int Np, void* S, const void* tw, cudaStream_t st);

// Work decomposition of the four step kernels.
struct Tiles {
  int rows;        // grid rows per block (row kernels)
  int conv_cols;   // spectrum slots per block (column convolution), or kConvThreePass
  int solve_cols;  // grid columns per block (y sweep)
};
// conv_cols value selecting the three-pass column convolution (conv3.cu)
constexpr int kConvThreePass = -1;

// Default work decomposition for FFT length Np; with N (the grid size) the
// row and column tiles are also capped so that a launch has about
// kSmallTileBlocks blocks or more where N allows it (small problems are
// latency-bound: spread them over the SMs).
constexpr int kSmallTileBlocks = 128;
template <typename T>
Tiles default_tiles(int Np, int N = 0);
template <typename T>
bool tiles_valid(const Geom& g, const Tiles& t);

template <typename T>
cudaError_t step_setup_attributes();

// FP32 register-FFT path (FFT length N' <= 1024; N' = 2048 for the dense
// form's FFT part).  One instance of a batch:
// natural-order tables and the in-place double-float state.
struct RegInst {
  const float2* tw1;    // [N'] two-level FFT twiddles exp(-2 pi i t k1 / N') at [k1 * TT + t]
  const float2* tw;     // [2N'] exp(-2 pi i k / 2N')
  const float2* lam_s;  // [N'] natural order, scaled as the bit-reversed tables
  const float2* lam_c;  // [N']
  const float* lreg;    // [(N'+1) * 2 * N'] symbol rows by x-frequency, even/odd halves, scaled
  const float* G;       // [N * r] border correction
  float* u_hi;          // state: u = u_hi + u_lo (double-float), u_d = u^n - u^{n-1}
  float* u_lo;
  float* u_d;
  const float* phi2;
  float2* S;            // spectrum scratch, slot-major: N' slots x N rows (S[k * N + row])
  float* W;             // N x N sweep scratch
  const float* F;       // optional source field (N x N) or nullptr
  float* C_hi;          // incremental remainder -kappa tau^2 L_h u^n (double-float)
  float* C_lo;
  unsigned short* Bh;   // dense-inverse form: BF16 split of B^n (ld ldp, zero-padded)
  unsigned short* Bl;
  int ldp;
  // dense form: the sweep GEMM's panel and tile counters (ndep ints), zeroed
  // by the B^n kernel for the GEMM launched after it (nullptr: none)
  int* dep;
  int ndep;
  int N, r;
  int ld;               // row pitch (elements) of the N x N arrays: u_hi, u_lo, u_d, phi2, W, F, C_hi, C_lo
  float tau, tau2;
  float fsc;            // time factor of the source for this step
  int gkind, first;
  float gc1, gc3, gcs;  // coefficients of g kind 3 (gc1 u + gc3 u^3 + gcs sin u)
  int eq;               // 0 wave, 1 diffusion (RhsParams::eq); tau2 = tau^2 or tau
};
constexpr int kMaxBatch = 32;
// passed by value as a __grid_constant__ kernel parameter (about 4 KB)
struct RegBatch {
  int count;
  RegInst in[kMaxBatch];
};
// whether a context of FFT length 2^logNp and precision prec (SADI_PREC_*)
// can step on the register path
bool reg_path_supported(int logNp, int prec);
// One step of every instance of the batch (all with FFT length 2^logNp);
// max_n = the largest N in the batch.  dense: only the row FFT, the column
// convolution and the B^n kernel run (events 0..2), the latter writing B^n to
// W and its BF16 split to Bh / Bl; the sweeps are left to the GEMMs.
cudaError_t launch_step_reg(const RegBatch& b, int logNp, int max_n, cudaStream_t st, cudaEvent_t* ev,
                            bool dense = false);
// natural-order FP32 tables of the register path from the FP64 setup products
cudaError_t run_reg_tables(const Geom& g, const double* lnat, double scale, const double2* lamc64,
                           const double2* lams64, float2* tw1, float* lreg, float2* lamc_nat, float2* lams_nat,
                           cudaStream_t st);

// One S-ADI step: u_next (may alias u_prev) from u_cur, u_prev.
// S: N x Np complex scratch, W: N x N scratch.
// ev (optional, 5 events): recorded before the first kernel and after each
// of the four kernels.  u_lo == nullptr: plain leapfrog u_next = 2u_cur - u_prev
// + uhat (u_next may alias u_prev).  u_lo != nullptr: compensated form, u_cur ==
// u_next = hi part, u_lo = lo part, u_prev = increment d, all in place.
// Ch, Cl (FP32 compensated form only, else nullptr): the incremental
// remainder C = -kappa tau^2 L_h u^n as a double-float pair, advanced in place
// by the convolution of the increment d = u_prev (the row FFT then reads d).
template <typename T>
cudaError_t launch_step(const Geom& g, const StepTables<T>& tb, const Tiles& tl, const RhsParams& rp, const T* u_cur,
                        T* u_prev, T* u_next, T* u_lo, const T* phi2, void* S, T* W, cudaStream_t st,
                        cudaEvent_t* ev = nullptr, float* Ch = nullptr, float* Cl = nullptr);
// C = -kappa tau^2 L_h u (N x N) into the double-float pair (Ch, Cl): the
// starting value of the incremental remainder (T = double gives it to FP64
// accuracy; needs the FP64 engine, N' <= 4096).
template <typename T>
cudaError_t launch_remainder(const Geom& g, const StepTables<T>& tb, const Tiles& tl, const T* u, void* S, float* Ch,
                             float* Cl, cudaStream_t st);

// Dense-inverse form on the shared-memory engine (FP32): row FFT of the
// increment d, column convolution, incremental remainder and B^n (events
// 0..2); B^n goes to W (N x N) and its BF16 split to Bh / Bl (ld ldp).
cudaError_t launch_dense_rows(const Geom& g, const StepTables<float>& tb, const Tiles& tl, const RhsParams& rp,
                              const float* u_cur, const float* d, const float* phi2, void* S, float* W, float* Ch,
                              float* Cl, unsigned short* Bh, unsigned short* Bl, int ldp, cudaStream_t st,
                              cudaEvent_t* ev);
// H^-1 - I of the N x N Toeplitz matrix H = I + s T(a_0 .. a_{N-1}) as a
// zero-padded npad x npad BF16 pair (Eh, El), from the generator c = H^-1 e_1
// (Durbin recursion) and the Gohberg-Semencul diagonal recurrence, in FP64.
// *status_host: 0 on success, 1 if the recursion broke down.
cudaError_t run_dense_inverse(const double* a1, int N, double s, int npad, void* Eh, void* El, int* status_host,
                              cudaStream_t st);

// ---- split-BF16 tensor-core GEMM, gemm_tc.cu ----------------------------------
// ACC = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T over K-major BF16 operands
// (row-major, K contiguous, zero-padded to whole tiles), then an epilogue.
// tile rows and K block; operands are padded to multiples of kTcTileN rows,
// which the 256-wide tiles and the 128-wide tiles of the GEMM both divide;
// every TMA box is kTcBox rows
constexpr int kTcTileM = 128, kTcTileN = 256, kTcTileK = 64, kTcBox = 128;
constexpr int kTcMaxBatch = 16;
enum TcMode { kTcStore = 0, kTcSweepX = 1, kTcSweepY = 2 };
struct TcEpi {
  int mode;
  int m_valid, n_valid;       // rows / columns of ACC that are written
  float* C;                   // kTcStore: out; kTcSweepX: B in, W out; kTcSweepY: W in (row-major, ld ldc)
  int ldc;
  unsigned short* t_hi;       // kTcSweepX: BF16 split of W^T (ld ldt), the next GEMM's B operand
  unsigned short* t_lo;
  int ldt;
  float* u_hi;                // kTcSweepY: double-float state and increment (ld ldu), updated in place
  float* u_lo;
  float* u_d;
  int ldu;
  int first;
  int* err;                   // set to 1 if a bounded wait of this problem's CTAs ran out (or nullptr)
  // 1: every row of C and of the state starts on a 16-byte boundary (ldc and
  // ldu multiples of 4, pointers 16-byte aligned) and the rows of the W^T
  // pair too (ldt a multiple of 8): the epilogue moves 16-byte vectors
  int vec;
};
// whether the epilogue of e may use 16-byte accesses (TcEpi::vec)
inline bool tc_vec_ok(const TcEpi& e) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  bool ok = e.ldc % 4 == 0 && al(e.C);
  if (e.mode == kTcSweepX) ok = ok && e.ldt % 8 == 0 && al(e.t_hi) && al(e.t_lo);
  if (e.mode == kTcSweepY) ok = ok && e.ldu % 4 == 0 && al(e.u_hi) && al(e.u_lo) && al(e.u_d);
  return ok;
}
struct TcInst {
  CUtensorMap a_hi, a_lo;     // A operand (M rows), box 128 x 64
  CUtensorMap b_hi, b_lo;     // B operand (N rows), box 128 x 64
  TcEpi e;
  int K;                      // padded contraction length (multiple of 64)
  int tiles_m, boxes_n;       // padded M / 128 and N / 128 of this problem
  // Order between problems of one launch (nullptr: none), by 128-column
  // panels: a tile of a problem with dep_wait starts (and reads its epilogue
  // inputs) once dep_wait[p] >= dep_need for each panel p of its B rows; a
  // problem with dep_signal adds 1 to dep_signal[p] for each panel p of a
  // tile's output columns once the tile's epilogue has stored it.  Waiting
  // problems must come after the problems they wait for in the launch.
  int* dep_wait;
  int dep_need;
  int* dep_signal;
};
// passed by value as a __grid_constant__ kernel parameter (about 10 KB)
struct TcBatch {
  int count;
  unsigned long long wait_ns;   // limit of every bounded wait of the launch (0: the default, 1 s)
  // zeroed int: with it the CTAs of a launch with 128-wide tiles take tiles
  // in order from this counter as they become free (nullptr: the static
  // order, CTA c taking tiles c, c + grid, ...)
  int* tile_next;
  // launched as a programmatic dependent of the kernel before it in the
  // stream (host-side choice; the kernel waits for that kernel after its
  // set-up in either case)
  int pdl;
  TcInst in[kTcMaxBatch];
};
// tensor map of a rows x kdim BF16 matrix (row-major) with box box_rows x 64
cudaError_t tc_encode(CUtensorMap* map, const void* base, int rows, int kdim, int box_rows);
// tensor maps and extents of one problem: A is M x K, B is N x K (padded sizes)
cudaError_t tc_set_operands(TcInst* in, const void* a_hi, const void* a_lo, const void* b_hi, const void* b_lo,
                            int M, int N, int K);
// one persistent launch for all b.count problems: at most one CTA per SM walks
// the output tiles of every problem, 128 x 256 tiles when they number at least
// two per SM (and every N is a multiple of 256), else 128 x 128; *err (or the
// problem's own e.err) set on a timed-out wait.  With dependencies between
// problems the launch is cooperative (every CTA resident at once).
cudaError_t launch_tc_gemm(const TcBatch& b, int* err, cudaStream_t st);
// FP32 rows x cols (ld src_ld) -> zero-padded prow x pcol BF16 hi / lo
cudaError_t launch_split_pad(const float* src, int rows, int cols, int src_ld, void* hi, void* lo, int prow, int pcol,
                             cudaStream_t st);

// ---- state watchdog, watchdog.cu ----------------------------------------------
// Device record of one context's watchdog: the last check's sum of u_ij^2
// (double) and its step, and a latched non-finite flag with the step of the
// first check that saw it (cleared by the host when the state is re-set).
constexpr int kWdMaxBlocks = 304;
struct WdState {
  double sumsq;
  long long step;
  int nonfinite;
  long long nonfinite_step;
  unsigned int ticket;              // blocks finished in the running launch (0 between launches)
  double partial[kWdMaxBlocks];
};
// sum of u[i]^2 over n elements (double or float) into wd, on stream st
cudaError_t launch_watchdog(const void* u, bool fp64, size_t n, WdState* wd, long long step, cudaStream_t st);

// ---- fixed scratch of sadi_step_noalloc, noalloc_scratch.cu ------------------
constexpr size_t kNoallocScratchBytes = size_t(32) << 20;
// Device address of the fixed scratch array on `device`, which must be the
// current device; looked up on the first call per device, cached afterwards.
cudaError_t noalloc_scratch_address(int device, void** out);

// ---- programmatic dependent launch of the shared-memory engine's kernels ------
// launch_dependent starts `kernel` on st as a programmatic dependent of the
// kernel before it in the stream: its blocks may be scheduled before that
// kernel has finished.  Every kernel launched this way opens with
// pdl_entry(), which lets the kernel after it be scheduled likewise and then
// waits until the kernel before it has completed and its writes are visible
// (a no-op for a launch without the attribute).  Every argument is passed
// explicitly (default arguments do not apply through the pointer).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    Args... args) {
  static_assert(sizeof...(KArgs) == sizeof...(Args), "every kernel argument passed explicitly");
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  a[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = a;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

}  // namespace sadi
