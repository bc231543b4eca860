// Fused batch path: one CTA decomposes one whole signal with the spectrum,
// the complex work array and the time-domain remainder resident in shared
// memory; CTAs pull signals from a global counter until the batch is done.
// HBM sees one read of the input and one write per IMF row and remainder.
#include "fif_device.cuh"
#include "fif_tc.cuh"

namespace fif {

// Per-signal loop state kept in shared memory rather than in registers: the
// kernel runs at 64 registers a thread, and values carried across the
// transforms and the m search would otherwise be spilled to local memory.
// Thread 0 writes it between barriers; every thread reads it after one.
struct LoopState {
  int K;         // IMFs extracted so far
  int flags;     // FIF_FLAG_* of the extracted IMFs
  int ek, ezc;   // extrema and zero crossings of the current remainder
  int etie;      // extrema tie of the current remainder
  float ermax;   // ||r||_inf of the current remainder
  float tau;     // tie band of the extrema count
  float sc;      // power-of-two scale of the spectrum for the m screen
};

struct FusedShared {
  FftSched S;
  RedScratch red;
  SigDesc d;
  LoopState ls;
  int sig;
  int ot[3];  // outer test result broadcast: reason, L, flags
};
static_assert(sizeof(FusedShared) + 16 <= kFusedHeader, "the fused kernel's shared header");

// One signal, Algorithm 2's outer loop with the inner loop replaced by the
// spectral multiplier (Theorem 5, eq. One step_algo).  TC: the inverse FFT's
// radix-16 passes run as split-BF16 tensor-core products (fif_tc.cuh; E = 16).
template <int E, bool TC>
__device__ void decompose_resident(FusedShared* sh, const MethodParams& mp,
                                   const float* __restrict__ signals, const Outputs& out,
                                   float2* spec, float2* work, float* rem, ffc* zf, float2* smtw) {
  const FftSched& S = sh->S;
  LoopState& ls = sh->ls;
  RedScratch* red = &sh->red;
  const int n = S.n, tid = threadIdx.x, nt = blockDim.x;

  if (smtw) {
    for (int u = tid; u < S.tw_entries; u += nt) {
      const float2 w = __ldg(&S.tw[u]);
      smtw[tw_slot(u)] = make_float2(w.x, -w.y);
    }
  }
  const TwSrc ts{smtw, S.tw, n, S.tw_fold, S.ptw};
  {
    const float* x = signals + sh->d.in_off;
    const float smax = forward_real<E>(x, rem, zf, spec, S, red);
    if (smax < 0.f) {  // NaN or Inf in the input
      float* orow = out.imfs + sh->d.out_off;
      for (int i = tid; i < n; i += nt) orow[i] = x[i];
      if (tid == 0) {
        const int sig = sh->d.idx;
        out.n_imfs[sig] = 0;
        out.sig_status[sig] = FIF_STOP_NONFINITE;
        if (out.diag) out.diag[(size_t)sig * (mp.max_imfs + 1)] = fif_imf_diag{0, 0, 0, 0.f};
      }
      return;
    }
    const float tau = tie_tau(smax);
    const ExtremaInfo e = count_extrema(rem, n, tau, red);
    if (tid == 0) {
      ls = LoopState{0, 0, e.k, e.zc, 0, e.rmax, tau, spectrum_scale(n, smax)};
      // (the input itself is exact on both sides: no extrema tie at step 0)
    }
    __syncthreads();
  }
  int reason = 0;
  for (;;) {
    // the outer test (binary64 division) on one thread, broadcast
    SpecPeak pk{0, 0};
    if (mp.peak_mask) pk = spectral_peak(spec, S, red);
    if (tid == 0) {
      const int sig = sh->d.idx;
      int L = 0, iflags = ls.etie ? FIF_FLAG_EXTREMA_TIE : 0;
      if (pk.tie) iflags |= FIF_FLAG_EXTREMA_TIE;
      sh->ot[0] = outer_test(ls.ek, ls.K, n, mp, out.mask_len + (size_t)sig * mp.max_imfs, L,
                             iflags, pk.k, S.ltab);
      sh->ot[1] = L;
      sh->ot[2] = iflags;
      if (out.diag) {
        fif_imf_diag* dg = out.diag + (size_t)sig * (mp.max_imfs + 1) + ls.K;
        dg->k_extrema = ls.ek;
        dg->zero_crossings = ls.ezc;
        if (sh->ot[0]) {
          dg->flags = iflags & FIF_FLAG_EXTREMA_TIE;
          dg->inf_norm = ls.ermax;
        }
      }
      if (sh->ot[0]) ls.flags |= iflags & FIF_FLAG_EXTREMA_TIE;
    }
    __syncthreads();
    reason = sh->ot[0];
    if (reason) break;
    const int L = sh->ot[1];
    int iflags = sh->ot[2];
    // m, the multiplier pairs of every bin in work, then IMF_hat and the spectral
    // remainder update applied inside the inverse real transform's split step
    const float2* msrc;
    const int m = select_m_mult(spec, work, S, L, mp, ls.sc, iflags, red, msrc);
    if constexpr (TC)
      inverse_real_mult_tc(spec, work, msrc, S, ts);
    else
      inverse_real_mult<E>(spec, work, msrc, S, ts);
    float* orow = out.imfs + sh->d.out_off + (size_t)ls.K * n;
    float imax, ermax;
    int ek, ezc, etie;
    if (!S.odd) {
      const EpiOut eo = epilogue_extrema_even(work, rem, orow, S, ls.tau, red);
      imax = eo.imax;
      ek = eo.k, ezc = eo.zc, etie = eo.tie, ermax = eo.rmax;
    } else {
      imax = store_imf_update_rem(work, rem, orow, S, red);
      const ExtremaInfo e = count_extrema(rem, n, ls.tau, red);
      ek = e.k, ezc = e.zc, etie = e.tie, ermax = e.rmax;
    }
    if (tid == 0) {
      const int sig = sh->d.idx, K = ls.K;
      out.m[(size_t)sig * mp.max_imfs + K] = m;
      if (!mp.force_L) out.mask_len[(size_t)sig * mp.max_imfs + K] = L;
      if (out.diag) {
        fif_imf_diag* dg = out.diag + (size_t)sig * (mp.max_imfs + 1) + K;
        dg->flags = iflags;
        dg->inf_norm = imax;
      }
      ls.flags |= iflags;
      ls.K = K + 1;
      ls.ek = ek, ls.ezc = ezc, ls.etie = etie, ls.ermax = ermax;
    }
    __syncthreads();
  }
  const int K = ls.K;
  float* rrow = out.imfs + sh->d.out_off + (size_t)K * n;
  for (int i = tid; i < n; i += nt) rrow[i] = rem[i];
  if (tid == 0) {
    const int sig = sh->d.idx;
    out.n_imfs[sig] = K;
    out.sig_status[sig] = reason | ls.flags;
  }
}

template <int E, bool TC>
__global__ void __launch_bounds__(E <= kWideMaxE ? 1024 : 512, 1) fused_kernel(const SigDesc* __restrict__ sigs, int nsig,
                                                    const FftSched* __restrict__ scheds,
                                                    MethodParams mp,
                                                    const float* __restrict__ signals, Outputs out,
                                                    int* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  FusedShared* sh = reinterpret_cast<FusedShared*>(smem);
  unsigned char* dyn = smem + kFusedHeader;
  for (;;) {
    if (threadIdx.x == 0) sh->sig = atomicAdd(counter, 1);
    __syncthreads();
    const int sig = sh->sig;
    if (sig >= nsig) break;
    if (threadIdx.x == 0) {
      sh->d = sigs[sig];
      sh->S = scheds[sh->d.sched];
    }
    __syncthreads();
    const FftSched& S = sh->S;
    float* rem = reinterpret_cast<float*>(dyn);
    float2* work = reinterpret_cast<float2*>(dyn + rem_bytes(S));
    float2* spec = work + work_points(S);
    ffc* zf = reinterpret_cast<ffc*>(dyn);
    float2* smtw = S.tw_shared ? spec + S.P : nullptr;
    decompose_resident<E, TC>(sh, mp, signals, out, spec, work, rem, zf, smtw);
    __syncthreads();
  }
}

#define FIF_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

static const void* fused_entry(int E, bool tc) {
  if (tc) return E == 16 ? (const void*)fused_kernel<16, true> : nullptr;
  switch (E) {
#define FIF_CASE(e) \
  case e:           \
    return (const void*)fused_kernel<e, false>;
    FIF_E_LIST(FIF_CASE)
#undef FIF_CASE
  }
  return nullptr;
}

int fused_blocks_per_sm(int E, int smem_bytes, int threads, bool tc) {
  const void* fn = fused_entry(E, tc);
  if (!fn) return 0;
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem_bytes) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_fused(int E, const SigDesc* d_sigs, int nsig, const FftSched* d_scheds,
                         int smem_bytes, int threads, int grid, const MethodParams& mp,
                         const float* signals, const Outputs& out, int* d_counter,
                         cudaStream_t st, bool tc) {
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (tc) {
    if (E != 16) return cudaErrorInvalidValue;
    fused_kernel<16, true><<<grid, threads, smem_bytes, st>>>(d_sigs, nsig, d_scheds, mp, signals,
                                                              out, d_counter);
    return cudaGetLastError();
  }
  switch (E) {
#define FIF_CASE(ee)                                                                            \
  case ee:                                                                                      \
    fused_kernel<ee, false><<<grid, threads, smem_bytes, st>>>(d_sigs, nsig, d_scheds, mp,      \
                                                               signals, out, d_counter);        \
    break;
    FIF_E_LIST(FIF_CASE)
#undef FIF_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fif
