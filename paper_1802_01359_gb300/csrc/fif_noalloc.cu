// fif_decompose_noalloc: the single-signal staged decomposition for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they decompose a
// signal: code on a latency-critical path (cudaMalloc synchronises the device
// and can take milliseconds), hosts that hand all device memory to their own
// pool up front, and plug-in style integrations that only permit allocation
// at start-up.  This entry point needs no plan: every array it uses besides
// the caller's inputs and outputs lives in one file-scope __device__ array of
// fixed size below.  The paper has no counterpart to this; it is a property
// of the library, not of the method.
//
// Each device that loads the library holds the array until the process exits.
// All calls share it and it keeps the last call's contents; every call
// rewrites what it reads before reading it (tables, spectrum, remainder, loop
// state).  Calls whose work overlaps on the GPU (other streams, or other host
// threads) race on the array: serialise them.
#include <math.h>
#include <string.h>

#include <mutex>

#include "fif_device.cuh"

namespace fif {

constexpr int kNoAllocMaxN = FIF_NOALLOC_MAX_N;
constexpr size_t kAlign = 256;
constexpr size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
// layout of the scratch array for any n <= kNoAllocMaxN
constexpr size_t kTwBytes = al(sizeof(float2) * kNoAllocMaxN);                // twiddles
constexpr size_t kSinBytes = al(sizeof(double) * (kNoAllocMaxN / 2 + 1));     // sin(pi t/n)
constexpr size_t kRowBytes = al(sizeof(float2) * (kNoAllocMaxN / 2 + 1));     // window row
constexpr size_t kSpecBytes = kRowBytes;                                       // spectrum
constexpr size_t kWorkBytes = al(sizeof(float2) * (kNoAllocMaxN + 2));         // work array
constexpr size_t kRemBytes = al(sizeof(float) * kNoAllocMaxN);                 // remainder
constexpr size_t kStateBytes = al(sizeof(int) * 16);
constexpr size_t kScratchBytes =
    2 * kTwBytes + kSinBytes + kRowBytes + kSpecBytes + kWorkBytes + kRemBytes + kStateBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NaScratch {
  float2* tw;
  float2* tw_lo;
  double* sin64;
  float2* row;
  float2* spec;
  float2* work;
  float* rem;
  int* state;
};

enum { NA_K = 0, NA_K_EXT, NA_ZC, NA_TIE, NA_FLAGS, NA_DONE, NA_L, NA_M, NA_IFLAGS, NA_SMAX, NA_RMAX };

template <int E>
__global__ void __launch_bounds__(512, 1) na_forward(FftSched S, const float* __restrict__ x,
                                                     NaScratch scr, Outputs out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch red;
  int* st = scr.state;
  const float smax = forward_real<E>(x, scr.rem, reinterpret_cast<ffc*>(smem), scr.spec, S, &red);
  if (smax < 0.f) {
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) out.imfs[i] = x[i];
    if (threadIdx.x == 0) {
      out.n_imfs[0] = 0;
      out.sig_status[0] = FIF_STOP_NONFINITE;
      if (out.diag) out.diag[0] = fif_imf_diag{0, 0, 0, 0.f};
      st[NA_DONE] = 1;
    }
    return;
  }
  const ExtremaInfo e = count_extrema(scr.rem, S.n, tie_tau(smax), &red);
  if (threadIdx.x == 0) {
    st[NA_K] = 0;
    st[NA_K_EXT] = e.k;
    st[NA_ZC] = e.zc;
    st[NA_TIE] = 0;
    st[NA_FLAGS] = 0;
    st[NA_DONE] = 0;
    st[NA_L] = 0;
    st[NA_SMAX] = __float_as_int(smax);
    st[NA_RMAX] = __float_as_int(e.rmax);
  }
}

// Outer-loop test; on a stop, writes the remainder row and the status.
__global__ void na_outer(FftSched S, NaScratch scr, Outputs out, MethodParams mp) {
  __shared__ RedScratch red;
  int* st = scr.state;
  if (st[NA_DONE]) return;
  const int K = st[NA_K], k = st[NA_K_EXT];
  int L = 0, iflags = st[NA_TIE] ? FIF_FLAG_EXTREMA_TIE : 0;
  SpecPeak pk{0, 0};
  if (mp.peak_mask) pk = spectral_peak(scr.spec, S, &red);
  if (pk.tie) iflags |= FIF_FLAG_EXTREMA_TIE;
  const int reason = outer_test(k, K, S.n, mp, out.mask_len, L, iflags, pk.k);
  if (out.diag && threadIdx.x == 0) {
    out.diag[K].k_extrema = k;
    out.diag[K].zero_crossings = st[NA_ZC];
  }
  if (reason) {
    float* rrow = out.imfs + (size_t)K * S.n;
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) rrow[i] = scr.rem[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      out.n_imfs[0] = K;
      out.sig_status[0] = reason | st[NA_FLAGS] | (iflags & FIF_FLAG_EXTREMA_TIE);
      if (out.diag) {
        out.diag[K].flags = iflags & FIF_FLAG_EXTREMA_TIE;
        out.diag[K].inf_norm = __int_as_float(st[NA_RMAX]);
      }
      st[NA_DONE] = 1;
    }
    return;
  }
  if (threadIdx.x == 0) {
    st[NA_L] = L;
    st[NA_IFLAGS] = iflags;
  }
}

// Window row {log2(1 - w_hat_k), w_hat_k} for the current L, in binary64 from
// the sine table (same values as the plan's table row).
__global__ void na_row(FftSched S, NaScratch scr) {
  const int* st = scr.state;
  if (st[NA_DONE]) return;
  const int L = st[NA_L];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < S.P) {
    const double w = what64(S, L, k);
    scr.row[k] = make_float2((float)(log1p(-w) * 1.4426950408889634), (float)w);
  }
}

// m selection on the current row: same search as select_m.
__global__ void __launch_bounds__(512, 1) na_select(FftSched S, NaScratch scr, MethodParams mp) {
  __shared__ RedScratch red;
  int* st = scr.state;
  if (st[NA_DONE]) return;
  const int L = st[NA_L];
  int iflags = st[NA_IFLAGS];
  const float sc = spectrum_scale(S.n, __int_as_float(st[NA_SMAX]));
  const int m = select_m_on_row(scr.spec, S, scr.row, L, mp, sc, iflags, &red);
  if (threadIdx.x == 0) {
    st[NA_M] = m;
    st[NA_IFLAGS] = iflags;
  }
}

__global__ void na_multiply(FftSched S, NaScratch scr, MethodParams mp) {
  const int* st = scr.state;
  if (st[NA_DONE]) return;
  const int m = st[NA_M], L = st[NA_L];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < S.P) {
    const float2 z = scr.spec[k];
    float g, omg;
    multiplier_th(m, __ldg(&scr.row[k]).x, S, L, k, mp, g, omg);
    scr.work[k] = make_float2(g * z.x, g * z.y);
    scr.spec[k] = make_float2(omg * z.x, omg * z.y);
  }
}

template <int E>
__global__ void __launch_bounds__(512, 1) na_inverse(FftSched S, NaScratch scr, Outputs out,
                                                     MethodParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch red;
  int* st = scr.state;
  if (st[NA_DONE]) return;
  float2* work = reinterpret_cast<float2*>(smem);
  float2* smtw = work + ((work_points(S) + 1) & ~(size_t)1);
  for (int k = threadIdx.x; k < S.P; k += blockDim.x) work[k] = scr.work[k];
  for (int u = threadIdx.x; u < S.tw_entries; u += blockDim.x) {
    const float2 w = __ldg(&S.tw[u]);
    smtw[tw_slot(u)] = make_float2(w.x, -w.y);
  }
  __syncthreads();
  const TwSrc ts{smtw, S.tw, S.n, S.tw_fold};
  inverse_real<E>(work, S, ts);
  const int K = st[NA_K];
  const float tau = tie_tau(__int_as_float(st[NA_SMAX]));
  float imax;
  ExtremaInfo e;
  if (!S.odd) {
    const EpiOut eo = epilogue_extrema_even(work, scr.rem, out.imfs + (size_t)K * S.n, S, tau, &red);
    imax = eo.imax;
    e = ExtremaInfo{eo.k, eo.zc, eo.tie, eo.rmax};
  } else {
    imax = store_imf_update_rem(work, scr.rem, out.imfs + (size_t)K * S.n, S, &red);
    e = count_extrema(scr.rem, S.n, tau, &red);
  }
  if (threadIdx.x == 0) {
    const int iflags = st[NA_IFLAGS];
    out.m[K] = st[NA_M];
    if (!mp.force_L) out.mask_len[K] = st[NA_L];
    if (out.diag) {
      out.diag[K].flags = iflags;
      out.diag[K].inf_norm = imax;
    }
    st[NA_FLAGS] |= iflags;
    st[NA_K] = K + 1;
    st[NA_K_EXT] = e.k;
    st[NA_ZC] = e.zc;
    st[NA_TIE] = e.tie;
    st[NA_RMAX] = __float_as_int(e.rmax);
  }
}

#define FIF_NA_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

template <int E>
static cudaError_t na_launch(const FftSched& s, const MethodParams& mp, const float* signal,
                             const Outputs& out, const NaScratch& scr, cudaStream_t st) {
  int dev = 0, maxsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const int dyn_max = maxsm - (int)sizeof(RedScratch);
  cudaFuncSetAttribute(na_forward<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  cudaFuncSetAttribute(na_inverse<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  const int threads = sched_threads(s);
  const size_t work_bytes = ((work_points(s) + 1) & ~(size_t)1) * sizeof(float2) +
                            tw_slots(s) * sizeof(float2);
  const size_t ff_bytes = (size_t)s.Nc * sizeof(ffc);
  const int pblocks = (s.P + 255) / 256;
  na_forward<E><<<1, threads, ff_bytes, st>>>(s, signal, scr, out);
  e = cudaGetLastError();
  for (int it = 0; e == cudaSuccess && it <= mp.max_imfs; it++) {
    na_outer<<<1, threads, 0, st>>>(s, scr, out, mp);
    na_row<<<pblocks, 256, 0, st>>>(s, scr);
    na_select<<<1, threads, 0, st>>>(s, scr, mp);
    na_multiply<<<pblocks, 256, 0, st>>>(s, scr, mp);
    na_inverse<E><<<1, threads, work_bytes, st>>>(s, scr, out, mp);
    e = cudaGetLastError();
  }
  return e;
}

// The address of g_noalloc_scratch on each device, taken once per device
// with that device current (the symbol's name is only a host-side stand-in).
static std::mutex g_setup_mu;
static void* g_scratch_addr[128];

static cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

cudaError_t build_twiddles(int n, float2* tw, float2* tw_lo, double* sin64, cudaStream_t st);

}  // namespace fif

using namespace fif;

static bool na_smooth(int64_t n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}
static_assert(kScratchBytes == FIF_NOALLOC_SCRATCH_BYTES, "the documented size of the scratch array");

extern "C" fif_status fif_decompose_noalloc(const fif_plan_desc* d, const float* signal, int64_t n,
                                            float* imfs, int32_t* m, int32_t* mask_len,
                                            int32_t* n_imfs, int32_t* sig_status,
                                            fif_imf_diag* diag, void* cuda_stream) {
  if (!d || !signal || !imfs || !n_imfs || !sig_status) return FIF_EINVAL;
  // a shape window needs a table per (n, L) that only a plan holds
  if (d->window == FIF_WIN_SHAPE) return FIF_EUNSUPPORTED;
  if (d->window != FIF_WIN_TRIANGLE || !(d->delta > 0.0) || !isfinite(d->delta) ||
      d->max_inner < 1 || d->max_inner > (1 << 20) || d->max_imfs < 0 || d->max_imfs > kMaxImfs ||
      (d->flags & ~(FIF_FORCE_L | FIF_APRIORI_N0 | FIF_PEAK_MASK)) ||
      !(d->gamma >= 0.0 && d->gamma < 1.0))
    return FIF_EINVAL;
  if (!(d->flags & FIF_FORCE_L) &&
      (!(d->nu > 0.0) || !isfinite(d->nu) || d->mask_scale < 1 || d->mask_scale > 2))
    return FIF_EINVAL;
  if (d->precision != FIF_PREC_FP32) return FIF_EUNSUPPORTED;
  if (d->max_imfs > 0 && (!m || !mask_len)) return FIF_EINVAL;
  if (n < 4) return FIF_EINVAL;
  if (n > kNoAllocMaxN || !na_smooth(n)) return FIF_EUNSUPPORTED;

  // schedule: the staged path's own (host arithmetic only, nothing allocated)
  FftSched s;
  if (!staged_schedule(n, s)) return FIF_EUNSUPPORTED;
  s.tw_shared = 1;

  cudaGetLastError();  // a pending error of earlier, unrelated work is not this call's
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return FIF_ECUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  NaScratch scr;
  scr.tw = reinterpret_cast<float2*>(b);
  b += kTwBytes;
  scr.tw_lo = reinterpret_cast<float2*>(b);
  b += kTwBytes;
  scr.sin64 = reinterpret_cast<double*>(b);
  b += kSinBytes;
  scr.row = reinterpret_cast<float2*>(b);
  b += kRowBytes;
  scr.spec = reinterpret_cast<float2*>(b);
  b += kSpecBytes;
  scr.work = reinterpret_cast<float2*>(b);
  b += kWorkBytes;
  scr.rem = reinterpret_cast<float*>(b);
  b += kRemBytes;
  scr.state = reinterpret_cast<int*>(b);
  s.tw = scr.tw;
  s.tw_lo = scr.tw_lo;
  s.sin64 = scr.sin64;
  s.wtab = scr.row;

  MethodParams mp;
  mp.nu = d->nu;
  mp.delta = d->delta;
  mp.delta2 = (float)(d->delta * d->delta);
  mp.mask_scale = d->mask_scale;
  mp.max_inner = d->max_inner;
  mp.max_imfs = d->max_imfs;
  mp.force_L = (d->flags & FIF_FORCE_L) ? 1 : 0;
  mp.apriori = (d->flags & FIF_APRIORI_N0) ? 1 : 0;
  mp.peak_mask = (d->flags & FIF_PEAK_MASK) ? 1 : 0;
  mp.threshold = d->gamma > 0.0 ? 1 : 0;
  mp.gamma = d->gamma;
  mp.log2_keep = d->gamma > 0.0 ? (float)log2(1.0 - d->gamma) : 0.f;
  Outputs out{imfs, m, mask_len, n_imfs, sig_status, diag};
  cudaStream_t st = (cudaStream_t)cuda_stream;

  e = build_twiddles(s.n, scr.tw, scr.tw_lo, scr.sin64, st);
  if (e == cudaSuccess) {
    switch (s.E) {
#define FIF_CASE(ee)                                   \
  case ee:                                             \
    e = na_launch<ee>(s, mp, signal, out, scr, st);    \
    break;
      FIF_NA_E_LIST(FIF_CASE)
#undef FIF_CASE
      default:
        e = cudaErrorInvalidValue;
    }
  }
  return e == cudaSuccess ? FIF_OK : FIF_ECUDA;
}
