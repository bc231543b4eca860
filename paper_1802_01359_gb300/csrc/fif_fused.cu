// Fused batch path: one CTA decomposes one whole signal with the spectrum,
// the complex work array and the time-domain remainder resident in shared
// memory; CTAs pull signals from a global counter until the batch is done.
// HBM sees one read of the input and one write per IMF row and remainder.
#include "fif_device.cuh"

namespace fif {

struct FusedShared {
  FftSched S;
  RedScratch red;
  int sig;
  int ot[3];  // outer test result broadcast: reason, L, flags
};
static_assert(sizeof(FusedShared) + 16 <= 1024, "fused_smem_bytes reserves 1 KiB for the header");

// One signal, Algorithm 2's outer loop with the inner loop replaced by the
// spectral multiplier (Theorem 5, eq. One step_algo).
template <int E>
__device__ void decompose_resident(const FftSched& S, const SigDesc& d, int sig,
                                   const MethodParams& mp, const float* __restrict__ signals,
                                   const Outputs& out, float2* spec, float2* work, float* rem,
                                   ffc* zf, float2* smtw, RedScratch* red, int* ot) {
  const int n = S.n, tid = threadIdx.x, nt = blockDim.x;
  const float* x = signals + d.in_off;
  float* orow = out.imfs + d.out_off;
  int32_t* m_out = out.m + (size_t)sig * mp.max_imfs;
  int32_t* L_io = out.mask_len + (size_t)sig * mp.max_imfs;
  fif_imf_diag* dg = out.diag ? out.diag + (size_t)sig * (mp.max_imfs + 1) : nullptr;

  if (smtw) {
    for (int u = tid; u < S.tw_entries; u += nt) {
      const float2 w = __ldg(&S.tw[u]);
      smtw[tw_slot(u)] = make_float2(w.x, -w.y);
    }
  }
  const TwSrc ts{smtw, S.tw, n, S.tw_fold};
  const float smax = forward_real<E>(x, rem, zf, spec, S, red);
  if (smax < 0.f) {  // NaN or Inf in the input
    for (int i = tid; i < n; i += nt) orow[i] = x[i];
    if (tid == 0) {
      out.n_imfs[sig] = 0;
      out.sig_status[sig] = FIF_STOP_NONFINITE;
      if (dg) dg[0] = fif_imf_diag{0, 0, 0, 0.f};
    }
    return;
  }
  const float tau = tie_tau(smax);
  const float sc = spectrum_scale(n, smax);
  ExtremaInfo e = count_extrema(rem, n, tau, red);
  e.tie = 0;  // the input itself is exact on both sides
  int K = 0, flags = 0, reason = 0;
  for (;;) {
    // the outer test (binary64 division) on one thread, broadcast
    int L = 0, iflags = e.tie ? FIF_FLAG_EXTREMA_TIE : 0;
    SpecPeak pk{0, 0};
    if (mp.peak_mask) pk = spectral_peak(spec, S, red);
    if (pk.tie) iflags |= FIF_FLAG_EXTREMA_TIE;
    if (tid == 0) {
      ot[0] = outer_test(e.k, K, n, mp, L_io, L, iflags, pk.k);
      ot[1] = L;
      ot[2] = iflags;
    }
    __syncthreads();
    reason = ot[0];
    L = ot[1];
    iflags = ot[2];
    if (dg && tid == 0) {
      dg[K].k_extrema = e.k;
      dg[K].zero_crossings = e.zc;
    }
    if (reason) {
      flags |= iflags & FIF_FLAG_EXTREMA_TIE;
      if (dg && tid == 0) {
        dg[K].flags = iflags & FIF_FLAG_EXTREMA_TIE;
        dg[K].inf_norm = e.rmax;
      }
      break;
    }
    const int m = select_m(spec, S, L, mp, sc, iflags, red);
    apply_multiplier(spec, work, S, L, m, mp);
    inverse_real<E>(work, S, ts);
    float imax;
    if (!S.odd) {
      const EpiOut eo = epilogue_extrema_even(work, rem, orow + (size_t)K * n, S, tau, red);
      imax = eo.imax;
      e = ExtremaInfo{eo.k, eo.zc, eo.tie, eo.rmax};
    } else {
      imax = store_imf_update_rem(work, rem, orow + (size_t)K * n, S, red);
      e = count_extrema(rem, n, tau, red);
    }
    if (tid == 0) {
      m_out[K] = m;
      if (!mp.force_L) L_io[K] = L;
      if (dg) {
        dg[K].flags = iflags;
        dg[K].inf_norm = imax;
      }
    }
    flags |= iflags;
    K++;
  }
  float* rrow = orow + (size_t)K * n;
  for (int i = tid; i < n; i += nt) rrow[i] = rem[i];
  if (tid == 0) {
    out.n_imfs[sig] = K;
    out.sig_status[sig] = reason | flags;
  }
}

template <int E>
__global__ void __launch_bounds__(E <= kWideMaxE ? 1024 : 512, 1) fused_kernel(const SigDesc* __restrict__ sigs, int nsig,
                                                    const FftSched* __restrict__ scheds,
                                                    MethodParams mp,
                                                    const float* __restrict__ signals, Outputs out,
                                                    int* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  FusedShared* sh = reinterpret_cast<FusedShared*>(smem);
  unsigned char* dyn = smem + 1024;
  for (;;) {
    if (threadIdx.x == 0) sh->sig = atomicAdd(counter, 1);
    __syncthreads();
    const int sig = sh->sig;
    if (sig >= nsig) break;
    const SigDesc d = sigs[sig];
    if (threadIdx.x == 0) sh->S = scheds[d.sched];
    __syncthreads();
    const FftSched& S = sh->S;
    float* rem = reinterpret_cast<float*>(dyn);
    float2* work = reinterpret_cast<float2*>(dyn + rem_bytes(S));
    float2* spec = work + work_points(S);
    ffc* zf = reinterpret_cast<ffc*>(dyn);
    float2* smtw = S.tw_shared ? spec + S.P : nullptr;
    decompose_resident<E>(S, d, d.idx, mp, signals, out, spec, work, rem, zf, smtw, &sh->red, sh->ot);
    __syncthreads();
  }
}

#define FIF_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

static const void* fused_entry(int E) {
  switch (E) {
#define FIF_CASE(e) \
  case e:           \
    return (const void*)fused_kernel<e>;
    FIF_E_LIST(FIF_CASE)
#undef FIF_CASE
  }
  return nullptr;
}

int fused_blocks_per_sm(int E, int smem_bytes, int threads) {
  const void* fn = fused_entry(E);
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
                         cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  switch (E) {
#define FIF_CASE(ee)                                                                     \
  case ee:                                                                               \
    fused_kernel<ee><<<grid, threads, smem_bytes, st>>>(d_sigs, nsig, d_scheds, mp, signals, \
                                                        out, d_counter);                 \
    break;
    FIF_E_LIST(FIF_CASE)
#undef FIF_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fif
