// Internal definitions shared by the host side and the kernels of libfif.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fif.h"

namespace fif {

constexpr int kMaxPass = 24;     // radix passes per FFT
constexpr int kEMax = 27;        // complex elements a thread holds during one FFT pass
constexpr int kMaxImfs = 64;
constexpr int kWideMaxE = 12;    // fused kernels with E <= kWideMaxE run up to 1024 threads

// FFT and table schedule for one signal length n = 2^a 3^b.
//   even n: the real transform is a complex FFT of Nc = n/2 points on
//           z_t = x_{2t} + i x_{2t+1}, plus an O(n) split step;
//   odd n:  a complex FFT of Nc = n points on the real data.
// Each FFT pass of radix R runs E/R butterflies per thread on T = Nc/E threads.
struct FftSched {
  int n;
  int Nc;
  int odd;
  int P;                       // spectrum bins kept: n/2+1 (even) or (n+1)/2 (odd)
  int E;
  int T;
  int npass;
  int radix[kMaxPass];
  int Lmax;                    // largest L with 2L-1 <= n
  int tw_fold;                 // symmetry folds of the shared twiddle table: 3 (octant, 8 | n),
                               // 2 (quarter, 4 | n), 1 (half, 2 | n), 0 (none)
  int tw_entries;              // entries of the shared twiddle table: n / 2^tw_fold + 1
                               // (stored in tw_slots() slots, see tw_slot)
  int tw_shared;               // 1 if the fused kernel keeps the table in shared memory
  int swz;                     // multi-pass FP32 levels: XOR mask of the swizzled column
                               // layout (work_slot, whole 16-point blocks), 0: plain
  const float2* tw;            // [n]  exp(-2 pi i t/n), rounded from binary64
  const float2* tw_lo;         // [n]  binary64 value minus tw, rounded (float-float twiddles)
  const float2* wtab;          // [Lmax * P]  row L-1: {log2(1 - w_hat_k), w_hat_k}
  const double* sin64;         // [n/2 + 1]  sin(pi t/n) in binary64
  const double* om64;          // shape window only: 1 - w_hat_k in binary64 at
                               // om64[(L-1) * om64_stride + k]; nullptr for the triangle
                               // (closed form from sin64)
  int om64_stride;             // P (plan table, a row per L) or 0 (one row, the current L)
  const float2* gtab;          // [Lmax * P] or nullptr: row L-1 holds {(1 - w_hat_k)^m,
                               // 1 - (1 - w_hat_k)^m} for m = max_inner (build_mult_table)
  const float2* ptw;           // [Nc - 1] or nullptr: the inverse FFT's per-pass twiddles for
                               // this schedule (build_pass_twiddles); nullptr: the folded table
  const int* ltab;             // [n + 1] or nullptr: ltab[k] = mask_scale * floor((nu * n) / k)
                               // for k >= 1 (binary64, the mask rule of the outer test), built
                               // on the host for the plan's nu and mask_scale
};

// Method parameters as the kernels see them.
struct MethodParams {
  double nu;
  double delta;
  float delta2;                // (float)(delta * delta), set on the host
  int mask_scale;
  int max_inner;
  int max_imfs;
  int force_L;
  int apriori;                 // m = the a-priori N0 of Theorem 5 instead of the search
  int threshold;               // gamma > 0: thresholded IMF (eq. I_gamma)
  double gamma;
  float log2_keep;             // (float) log2(1 - gamma), set on the host
  int peak_mask;               // L from the spectral peak instead of the extrema count
};

// One signal of a batch launch.
struct SigDesc {
  int64_t in_off;
  int64_t out_off;
  int sched;                   // index into the schedule array
  int n;
  int idx;                     // signal index in the caller's batch (output row)
  int pad;
};

struct Outputs {
  float* imfs;
  int32_t* m;
  int32_t* mask_len;
  int32_t* n_imfs;
  int32_t* sig_status;
  fif_imf_diag* diag;
};

// Shared-memory layout of the fused kernel after a 1 KiB header: the
// time-domain remainder (n floats, padded to 16 bytes), the complex work array
// (Nc+1 points for even n, n for odd n) and the spectrum (P points).  The
// float-float forward transform (16 bytes per point, Nc points) overlays the
// first two regions (and, for odd n, the start of the third, which it does
// not read back).
__host__ __device__ inline size_t rem_bytes(const FftSched& s) { return ((size_t)s.n * sizeof(float) + 15) & ~(size_t)15; }
// Bytes of the fused kernel's shared header (schedule, reduction scratch,
// loop state) ahead of its arrays.
constexpr size_t kFusedHeader = 1280;
__host__ __device__ inline size_t work_points(const FftSched& s) { return (size_t)(s.odd ? s.n : s.Nc + 1); }
// Slot of entry u of a shared twiddle table: u with its low four bits XOR-ed
// by a fold of its higher bits.  The passes of a transform read entries a
// power of two apart (k times n / (Ns R), folded); without the swizzle those
// land in one bank (up to 32-way conflicts).  A bijection inside each block of
// 16 entries, so consecutive entries still hit distinct banks.
__host__ __device__ inline int tw_slot(int u) {
  const int x = u >> 4;
  return u ^ ((x ^ (x >> 4) ^ (x >> 8) ^ (x >> 12)) & 15);
}
// Slots a table of s.tw_entries entries occupies (whole blocks of 16).
__host__ __device__ inline size_t tw_slots(const FftSched& s) {
  return ((size_t)s.tw_entries + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t tw_table_bytes(const FftSched& s) {
  return s.tw_shared ? tw_slots(s) * sizeof(float2) : 0;
}
inline size_t fused_smem_bytes(const FftSched& s) {
  return kFusedHeader + rem_bytes(s) + (work_points(s) + (size_t)s.P) * sizeof(float2) +
         tw_table_bytes(s);
}

inline int sched_threads(const FftSched& s) {
  int t = s.T < 128 ? 128 : s.T;
  if (s.n <= 256 && t > 64) t = 64;
  return (t + 31) & ~31;
}

// ---- large-signal path (fif_large.cu) ----
// The complex FFT of Nc = R1 R2 points runs as two passes through global
// memory, each a set of shared-memory sub-FFTs of R1 (then R2) points.
struct LgSched {
  FftSched S;             // the signal length: n, Nc, odd, P, Lmax, tw/tw_lo over n, sin64
  FftSched S1, S2;        // complex sub-FFTs of R1 and R2 points (n = Nc = R): the FP32 inverse levels
  FftSched F1, F2;        // the same sub-FFTs for the float-float forward levels (the fixed
                          // rule's schedules; the tuner changes S1 and S2 only)
  int R1, R2;
  int TJ1, TJ2;           // sub-FFTs per CTA in the FP32 passes
  int TJF1, TJF2;         // sub-FFTs per CTA in the float-float passes
  int B, Bs;              // W^m = thi[m >> Bs] * tlo[m & (B - 1)], B = 2^Bs, W = exp(-2 pi i / Nc)
  const float2* thi;
  const float2* thi_lo;
  const float2* tlo;
  const float2* tlo_lo;
  const float2* sinff;    // {hi, lo} of sin(pi t/n), t = 0..n/2
  const float2* rcpff;    // {hi, lo} of 1/sin(pi k/n), k = 1..n/2 (entry 0 unused)
  int sel_blocks;         // CTAs per signal in the grid-wide m search
  const double* shape;    // shape window: the shape's samples (device); nullptr: triangle
  int shape_len;
  int tc1, tc2;           // FIF_PREC_SPLIT_BF16: the FP32 inverse level runs its radix-16 passes
                          // on the tensor cores (sub-FFT schedule E = 16, T a multiple of 32)
};

// The grid-wide m search evaluates SD_j at up to kSelCand values of j per
// round; each CTA leaves one partial per candidate (kSelPartBytes each, FP32
// screen and binary64 tie-break side by side).
constexpr int kSelCand = 8;
// Points of padding between the columns of an FP32 level tile in shared memory.
constexpr int kLgColPad = 4;
constexpr int kSelBlocksMax = 1024;
constexpr int kSelPartBytes = 48;
constexpr int kLgStateWords = 32;

// One signal of a large-length class: offsets into the caller's arrays and
// the signal's working arrays (za/zb hold float-float complex points, 16
// bytes each, during the forward transform).
struct LgSig {
  int64_t in_off;
  int64_t out_off;
  int idx;                // signal index in the batch (rows of m, mask_len, ...)
  int pad;
  float4* za;
  float4* zb;
  float2* spec;
  float2* work;
  float2* work2;
  float* rem;             // remainder of even iterations (and the input copy)
  float* rem2;            // remainder of odd iterations
  float2* row;
  int* st;                // kLgStateWords state words, zeroed before each run
  unsigned char* part;    // sel_blocks * kSelCand * kSelPartBytes
  double* om64;           // shape window: 1 - w_hat_k of the current L in binary64 [P]
};

cudaError_t large_build_tables(const LgSched& G, float2* thi, float2* thi_lo, float2* tlo,
                               float2* tlo_lo, float2* sinff, float2* rcpff, cudaStream_t st);
cudaError_t large_run(const LgSched& G, const LgSig* d_sigs, int nsig, const MethodParams& mp,
                      const float* signals, const Outputs& out, cudaStream_t st);
size_t large_level_smem(const LgSched& G, int level, bool ff);
cudaError_t large_set_attrs(const LgSched& G);
int large_sel_rounds(int max_inner);
// Kernel launches large_run enqueues for nsig signals of one class.
int large_launches(int nsig, const MethodParams& mp, bool shape);

// The schedule the staged path uses for length n (at most 512 threads, the
// folded twiddle table in shared memory): FFT radix passes, E, T, P, Lmax.
// Host arithmetic only, no allocation.  false if n is not 2^a 3^b in
// [4, 2^24] or no schedule exists.
bool staged_schedule(int64_t n, FftSched& s);

// Kernel launchers (fif_fused.cu, fif_staged.cu, fif_tables.cu).
// tc: the split-BF16 tensor-core variant of the inverse FFT (E = 16 only).
cudaError_t launch_fused(int E, const SigDesc* d_sigs, int nsig, const FftSched* d_scheds,
                         int smem_bytes, int threads, int grid, const MethodParams& mp,
                         const float* signals, const Outputs& out, int* d_counter,
                         cudaStream_t st, bool tc = false);
int fused_blocks_per_sm(int E, int smem_bytes, int threads, bool tc = false);

struct StagedScratch {
  float2* spec;   // [P]
  float2* work;   // [max(Nc+1, n)]
  float* rem;     // [n]
  int* state;     // per-signal loop state
};
cudaError_t launch_staged(const FftSched& s, const FftSched* d_sched, const MethodParams& mp,
                          const float* signal, const Outputs& out, const StagedScratch& scr,
                          cudaStream_t st);

// {(1 - w_hat_k)^m, 1 - (1 - w_hat_k)^m} for every L = 1..Lmax and bin k < P in
// binary64, rounded (bins passing whole under gamma > 0 get {1, 0}); om64:
// the shape window's rows of 1 - w_hat, or nullptr for the triangle.
cudaError_t build_mult_table(int n, int P, int Lmax, int m, double gamma, const double* om64,
                             float2* gtab, cudaStream_t st);
// The radices of a schedule, passed by value to the table kernel.
struct PassRadix {
  int r[kMaxPass];
};
// Per-pass twiddles of schedule s for its inverse FFT (s.tw must be built):
// ptw[(Ns - 1) + (r - 1) Ns + k] = exp(+2 pi i r k/(Ns R)) for the pass of
// radix R after Ns points, Nc - 1 entries in all.
cudaError_t build_pass_twiddles(const FftSched& s, float2* ptw, cudaStream_t st);
cudaError_t build_tables(int n, int P, int Lmax, float2* tw, float2* tw_lo, float2* wtab,
                         double* sin64, cudaStream_t st);
cudaError_t build_twiddles(int n, float2* tw, float2* tw_lo, double* sin64, cudaStream_t st);
// Window rows of a shape-generated window for every L = 1..s.Lmax into wtab
// and om64 (s.tw / s.tw_lo must be built); g: device copy of the shape.
cudaError_t build_shape_window(const FftSched& s, const double* g, int glen, float2* wtab,
                               double* om64, cudaStream_t st);

}  // namespace fif
