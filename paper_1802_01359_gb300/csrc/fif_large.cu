// Large-signal path: lengths whose spectrum, work array and remainder do not
// fit one CTA's shared memory (up to n = 2^24 and beyond).  Every step is a
// kernel over all signals of one length class (grid y = signal):
//   pack      float-float packing of the input, r = s, max |s|, NaN check
//   level 1/2 complex FFT of Nc = R1 R2 points as two passes through global
//             memory; each CTA runs TJ shared-memory sub-FFTs of R points on
//             TJ adjacent columns (coalesced 32-byte runs), the second pass
//             first multiplies by W_Nc^(r k) (the four-step form of the
//             Stockham factorisation with radices R1 and R2)
//   split     real-transform split, rounded once to the FP32 spectrum
// then per outer iteration:
//   ctl       one CTA per signal: extrema count of r, bookkeeping of the last
//             IMF, outer-loop test (Algorithm 2); on a stop the remainder row
//   row       window eigenvalues {log2(1-w_hat_k), w_hat_k} for this L, in
//             float-float from sine and reciprocal-sine tables
//   select    one CTA per signal: m by eq. SD (FP32 screen, binary64 tie-break)
//   multiply  IMF_hat = (1-w_hat)^m r_hat, r_hat <- (1 - (1-w_hat)^m) r_hat
//   presplit  inverse real-transform split
//   level 1/2 inverse complex FFT
//   epilogue  IMF row = C2R / n, r <- r - IMF
#include "fif_device.cuh"

namespace fif {

enum {
  LG_K = 0, LG_KEXT, LG_ZC, LG_TIE, LG_FLAGS, LG_DONE, LG_L, LG_M, LG_IFLAGS, LG_SMAX, LG_RMAX,
  LG_BAD, LG_IMAX
};

// The caller's arrays of one signal.
struct LgIO {
  const float* x;
  float* out;
  int32_t* m;
  int32_t* mask_len;
  int32_t* n_imfs;
  int32_t* status;
  fif_imf_diag* diag;
};

__device__ __forceinline__ LgIO lg_io(const LgSig& sg, const float* signals, const Outputs& o,
                                      int K) {
  LgIO io;
  io.x = signals + sg.in_off;
  io.out = o.imfs + sg.out_off;
  io.m = o.m + (size_t)sg.idx * K;
  io.mask_len = o.mask_len + (size_t)sg.idx * K;
  io.n_imfs = o.n_imfs + sg.idx;
  io.status = o.sig_status + sg.idx;
  io.diag = o.diag ? o.diag + (size_t)sg.idx * (K + 1) : nullptr;
  return io;
}

// W_Nc^m (forward sign), 0 <= m < Nc
template <class Cx, bool INV>
__device__ __forceinline__ Cx inter_twiddle(const LgSched& G, int m);
template <>
__device__ __forceinline__ float2 inter_twiddle<float2, false>(const LgSched& G, int m) {
  const int a = m / G.B, b = m - a * G.B;
  return cmul(__ldg(&G.thi[a]), __ldg(&G.tlo[b]));
}
template <>
__device__ __forceinline__ float2 inter_twiddle<float2, true>(const LgSched& G, int m) {
  return cconj(inter_twiddle<float2, false>(G, m));
}
template <>
__device__ __forceinline__ ffc inter_twiddle<ffc, false>(const LgSched& G, int m) {
  const int a = m / G.B, b = m - a * G.B;
  const float2 h1 = __ldg(&G.thi[a]), l1 = __ldg(&G.thi_lo[a]);
  const float2 h2 = __ldg(&G.tlo[b]), l2 = __ldg(&G.tlo_lo[b]);
  return cmul(ffc{ff{h1.x, l1.x}, ff{h1.y, l1.y}}, ffc{ff{h2.x, l2.x}, ff{h2.y, l2.y}});
}
template <>
__device__ __forceinline__ ffc inter_twiddle<ffc, true>(const LgSched& G, int m) {
  return cconj(inter_twiddle<ffc, false>(G, m));
}

__device__ __forceinline__ int first_signal_point(int& step) {
  step = gridDim.x * blockDim.x;
  return blockIdx.x * blockDim.x + threadIdx.x;
}

// ------------------------------------------------------------ forward

__global__ void lg_pack(const LgSig* __restrict__ sigs, LgSched G, const float* __restrict__ signals) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.y];
  const float* x = signals + sg.in_off;
  const int n = G.S.n, Nc = G.S.Nc;
  ffc* za = reinterpret_cast<ffc*>(sg.za);
  float amax = 0.f;
  int bad = 0, step;
  for (int t = first_signal_point(step); t < Nc; t += step) {
    float a, b;
    if (!G.S.odd) {
      a = x[2 * t];
      b = x[2 * t + 1];
      sg.rem[2 * t] = a;
      sg.rem[2 * t + 1] = b;
      za[t] = ffc{ff{a, 0.f}, ff{b, 0.f}};
    } else {
      a = x[t];
      b = 0.f;
      sg.rem[t] = a;
      za[t] = ffc{ff{a, 0.f}, ff{0.f, 0.f}};
    }
    amax = fmaxf(amax, fmaxf(fabsf(a), fabsf(b)));
    bad |= !isfinite(a) || !isfinite(b);
  }
  bad = __syncthreads_or(bad);
  float dummy = 0.f;
  block_reduce2(amax, dummy, OpMax(), 0.f, &red);
  if (threadIdx.x == 0) {
    atomicMax(&sg.st[LG_SMAX], __float_as_int(amax));  // non-negative floats order as ints
    if (bad) atomicOr(&sg.st[LG_BAD], 1);
  }
}

// One pass of TJ sub-FFTs of R points per CTA.  LV 1: butterflies j (Ns = 1)
// read x[j + r Nc/R1], write y[j R1 + r].  LV 2: butterflies j = k < R1
// (Ns = R1) read y[j + r R1] times W^(r j), write z[j + r R1].
template <class Cx, bool INV, int E, int LV>
__global__ void __launch_bounds__(512, 1) lg_level(const LgSig* __restrict__ sigs, LgSched G) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LgSig sg = sigs[blockIdx.y];
  if (INV && sg.st[LG_DONE]) return;
  constexpr bool FF = sizeof(Cx) == 16;
  const FftSched& SR = LV == 1 ? G.S1 : G.S2;
  const int R = LV == 1 ? G.R1 : G.R2;
  const int TJ = FF ? (LV == 1 ? G.TJF1 : G.TJF2) : (LV == 1 ? G.TJ1 : G.TJ2);
  const int stride_in = LV == 1 ? G.R2 : G.R1;
  const Cx* in;
  Cx* out;
  if (FF) {
    in = reinterpret_cast<const Cx*>(LV == 1 ? sg.za : sg.zb);
    out = reinterpret_cast<Cx*>(LV == 1 ? sg.zb : sg.za);
  } else {
    in = reinterpret_cast<const Cx*>(LV == 1 ? sg.work2 : sg.work);
    out = reinterpret_cast<Cx*>(LV == 1 ? sg.work : sg.work2);
  }
  Cx* buf = reinterpret_cast<Cx*>(smem);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int j0 = blockIdx.x * TJ;
  for (int f = tid; f < TJ * R; f += nt) {
    const int r = f / TJ, g = f - r * TJ;
    Cx v = in[j0 + g + r * stride_in];
    if (LV == 2) v = cmul(v, inter_twiddle<Cx, INV>(G, r * (j0 + g)));
    buf[g * R + r] = v;
  }
  float2* q = nullptr;
  if constexpr (!FF) {
    q = reinterpret_cast<float2*>(smem + (size_t)TJ * R * sizeof(Cx));
    for (int u = tid; u < SR.tw_entries; u += nt) {
      const float2 w = __ldg(&SR.tw[u]);
      q[u] = make_float2(w.x, -w.y);
    }
  }
  __syncthreads();
  const int T = SR.T, g = tid / T;
  const int lt = g < TJ ? tid - g * T : T;  // T: inactive in the sub-FFT
  Cx* mine = buf + (size_t)(g < TJ ? g : 0) * R;
  if constexpr (FF) {
    fft_inplace<Cx, INV, E>(mine, SR, SR, lt);
  } else {
    const TwSrc ts{q, SR.tw, SR.n, SR.tw_fold};
    fft_inplace<Cx, INV, E>(mine, SR, ts, lt);
  }
  if (LV == 1) {
    for (int f = tid; f < TJ * R; f += nt) {
      const int gg = f / R, r = f - gg * R;
      out[(size_t)(j0 + gg) * R + r] = buf[f];
    }
  } else {
    for (int f = tid; f < TJ * R; f += nt) {
      const int r = f / TJ, gg = f - r * TJ;
      out[j0 + gg + r * G.R1] = buf[gg * R + r];
    }
  }
}

// Real-transform split (same formulas as forward_real), rounded once.
__global__ void lg_split_fwd(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  const ffc* za = reinterpret_cast<const ffc*>(sg.za);
  const int Nc = G.S.Nc;
  int step;
  if (!G.S.odd) {
    for (int k = first_signal_point(step); k <= Nc / 2; k += step) {
      const ffc zk = za[k];
      const ffc zc = cconj(za[k == 0 ? 0 : Nc - k]);
      const ffc e = chalf(cadd(zk, zc));
      const ffc o = rot_i<false>(chalf(csub(zk, zc)));
      const ffc wo = cmul(load_tw<ffc, false>(G.S, k), o);
      const ffc xk = cadd(e, wo);
      const ffc xc = cconj(csub(e, wo));
      sg.spec[k] = make_float2(xk.re.hi, xk.im.hi);
      sg.spec[Nc - k] = make_float2(xc.re.hi, xc.im.hi);
    }
  } else {
    for (int k = first_signal_point(step); k < G.S.P; k += step)
      sg.spec[k] = make_float2(za[k].re.hi, za[k].im.hi);
  }
}

// ------------------------------------------------------------ per IMF

__global__ void __launch_bounds__(512, 1) lg_ctl(const LgSig* __restrict__ sigs, LgSched G,
                                                 MethodParams mp, int it,
                                                 const float* __restrict__ signals, Outputs o) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.x];
  const LgIO io = lg_io(sg, signals, o, mp.max_imfs);
  int* st = sg.st;
  if (st[LG_DONE]) return;
  const int n = G.S.n, tid = threadIdx.x, nt = blockDim.x;
  if (it == 0 && st[LG_BAD]) {
    for (int i = tid; i < n; i += nt) io.out[i] = io.x[i];
    if (tid == 0) {
      io.n_imfs[0] = 0;
      io.status[0] = FIF_STOP_NONFINITE;
      if (io.diag) io.diag[0] = fif_imf_diag{0, 0, 0, 0.f};
      st[LG_DONE] = 1;
    }
    return;
  }
  const float tau = tie_tau(__int_as_float(st[LG_SMAX]));
  ExtremaInfo e = count_extrema(sg.rem, n, tau, &red);
  int K = st[LG_K];
  int flags = st[LG_FLAGS];
  if (it > 0) {  // the IMF extracted in the previous iteration
    const int iflags = st[LG_IFLAGS];
    if (tid == 0) {
      io.m[K] = st[LG_M];
      if (!mp.force_L) io.mask_len[K] = st[LG_L];
      if (io.diag) {
        io.diag[K].flags = iflags;
        io.diag[K].inf_norm = __int_as_float(st[LG_IMAX]);
      }
    }
    flags |= iflags;
    K++;
  } else {
    e.tie = 0;  // the input itself is exact on both sides
  }
  int L = 0, iflags = e.tie ? FIF_FLAG_EXTREMA_TIE : 0;
  const int reason = outer_test(e.k, K, n, mp, io.mask_len, L, iflags);
  if (io.diag && tid == 0) {
    io.diag[K].k_extrema = e.k;
    io.diag[K].zero_crossings = e.zc;
  }
  if (reason) {
    float* rrow = io.out + (size_t)K * n;
    for (int i = tid; i < n; i += nt) rrow[i] = sg.rem[i];
    if (tid == 0) {
      flags |= iflags & FIF_FLAG_EXTREMA_TIE;
      io.n_imfs[0] = K;
      io.status[0] = reason | flags;
      if (io.diag) {
        io.diag[K].flags = iflags & FIF_FLAG_EXTREMA_TIE;
        io.diag[K].inf_norm = e.rmax;
      }
      st[LG_K] = K;
      st[LG_FLAGS] = flags;
      st[LG_DONE] = 1;
    }
    return;
  }
  if (tid == 0) {
    st[LG_K] = K;
    st[LG_FLAGS] = flags;
    st[LG_L] = L;
    st[LG_IFLAGS] = iflags;
    st[LG_IMAX] = 0;
  }
}

// x / L in float-float for an integer 1 <= L < 2^24 (exact in binary32)
__device__ __forceinline__ ff ff_div_int(ff x, int L) {
  const float fl = (float)L;
  const float q1 = __fdiv_rn(x.hi, fl);
  const float r = __fadd_rn(__fmaf_rn(-q1, fl, x.hi), x.lo);
  const float q2 = __fdiv_rn(r, fl);
  const float hi = __fadd_rn(q1, q2);
  return ff{hi, __fsub_rn(q2, __fsub_rn(hi, q1))};
}

// Window eigenvalues for this IMF's L: w_hat_k = [sin(pi k L/n) / (L sin(pi k/n))]^2
// (eq. Lambdas for the sampled triangle) in float-float, then rounded:
// row[k] = {log2(1 - w_hat_k), w_hat_k}.
__global__ void lg_row(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  const int L = sg.st[LG_L];
  const int n = G.S.n;
  int step;
  for (int k = first_signal_point(step); k < G.S.P; k += step) {
    float hl, wf;
    if (k == 0) {
      hl = -INFINITY;
      wf = 1.f;
    } else {
      long long t = ((long long)k * (long long)L) % n;
      if (t > n - t) t = n - t;
      const float2 sv = __ldg(&G.sinff[t]), rv = __ldg(&G.rcpff[k]);
      const ff x = ff_mul(ff{sv.x, sv.y}, ff{rv.x, rv.y});
      const ff q = ff_div_int(x, L);
      ff w = ff_mul(q, q);
      if (w.hi >= 1.f) w = ff{1.f, 0.f};
      wf = w.hi;
      if (wf <= 0.5f) {
        hl = log1pf(-wf) * 1.44269504088896341f;
      } else {
        const ff omw = ff_sub(ff{1.f, 0.f}, w);
        hl = omw.hi > 0.f ? log2f(omw.hi) : -INFINITY;
      }
    }
    sg.row[k] = make_float2(hl, wf);
  }
}

__global__ void __launch_bounds__(512, 1) lg_select(const LgSig* __restrict__ sigs, LgSched G,
                                                    MethodParams mp) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.x];
  int* st = sg.st;
  if (st[LG_DONE]) return;
  const int L = st[LG_L];
  int iflags = st[LG_IFLAGS];
  const float sc = spectrum_scale(G.S.n, __int_as_float(st[LG_SMAX]));
  const int m = select_m_on_row(sg.spec, G.S, sg.row, L, mp, sc, iflags, &red);
  if (threadIdx.x == 0) {
    st[LG_M] = m;
    st[LG_IFLAGS] = iflags;
  }
}

__global__ void lg_multiply(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  const int m = sg.st[LG_M];
  int step;
  for (int k = first_signal_point(step); k < G.S.P; k += step) {
    const float2 z = sg.spec[k];
    float g, omg;
    multiplier(m, sg.row[k].x, g, omg);
    sg.work[k] = make_float2(g * z.x, g * z.y);
    sg.spec[k] = make_float2(omg * z.x, omg * z.y);
  }
}

// Inverse real-transform split (same formulas as inverse_real), work -> work2.
__global__ void lg_presplit(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  const int Nc = G.S.Nc, n = G.S.n;
  int step;
  if (!G.S.odd) {
    for (int k = first_signal_point(step); k <= Nc / 2; k += step) {
      const float2 xk = sg.work[k];
      const float2 xc = sg.work[Nc - k];
      const float2 f = make_float2(xk.x + xc.x, xk.y - xc.y);
      const float2 g = make_float2(xk.x - xc.x, xk.y + xc.y);
      const float2 wg = cmul(cconj(__ldg(&G.S.tw[k])), g);
      const float2 iwg = make_float2(-wg.y, wg.x);
      sg.work2[k] = cadd(f, iwg);
      if (k != 0) sg.work2[Nc - k] = cconj(csub(f, iwg));
    }
  } else {
    for (int k = first_signal_point(step); k < G.S.P; k += step) {
      const float2 v = sg.work[k];
      sg.work2[k] = v;
      if (k != 0) sg.work2[n - k] = cconj(v);
    }
  }
}

__global__ void lg_epilogue(const LgSig* __restrict__ sigs, LgSched G, float* __restrict__ imfs) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  const int n = G.S.n, K = sg.st[LG_K];
  const float inv_n = 1.f / (float)n;
  float* orow = imfs + sg.out_off + (size_t)K * n;
  float imax = 0.f;
  int step;
  if (!G.S.odd) {
    for (int t = first_signal_point(step); t < G.S.Nc; t += step) {
      const float2 z = sg.work2[t];
      const float a = z.x * inv_n, b = z.y * inv_n;
      orow[2 * t] = a;
      orow[2 * t + 1] = b;
      sg.rem[2 * t] -= a;
      sg.rem[2 * t + 1] -= b;
      imax = fmaxf(imax, fmaxf(fabsf(a), fabsf(b)));
    }
  } else {
    for (int t = first_signal_point(step); t < n; t += step) {
      const float a = sg.work2[t].x * inv_n;
      orow[t] = a;
      sg.rem[t] -= a;
      imax = fmaxf(imax, fabsf(a));
    }
  }
  float dummy = 0.f;
  block_reduce2(imax, dummy, OpMax(), 0.f, &red);
  if (threadIdx.x == 0) atomicMax(&sg.st[LG_IMAX], __float_as_int(imax));
}

// ------------------------------------------------------------ tables

__global__ void lg_table_kernel(LgSched G, float2* thi, float2* thi_lo, float2* tlo,
                                float2* tlo_lo, float2* sinff, float2* rcpff) {
  const int Nc = G.S.Nc, n = G.S.n, B = G.B;
  const int nhi = (Nc + B - 1) / B;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s, c;
  if (i < nhi) {
    sincospi(2.0 * (double)((long long)i * B) / (double)Nc, &s, &c);
    const float ch = (float)c, sh = (float)(-s);
    thi[i] = make_float2(ch, sh);
    thi_lo[i] = make_float2((float)(c - (double)ch), (float)(-s - (double)sh));
  }
  if (i < B) {
    sincospi(2.0 * (double)i / (double)Nc, &s, &c);
    const float ch = (float)c, sh = (float)(-s);
    tlo[i] = make_float2(ch, sh);
    tlo_lo[i] = make_float2((float)(c - (double)ch), (float)(-s - (double)sh));
  }
  if (i <= n / 2) {
    const double v = sinpi((double)i / (double)n);
    const float vh = (float)v;
    sinff[i] = make_float2(vh, (float)(v - (double)vh));
    if (i > 0) {
      const double r = 1.0 / v;
      const float rh = (float)r;
      rcpff[i] = make_float2(rh, (float)(r - (double)rh));
    } else {
      rcpff[0] = make_float2(0.f, 0.f);
    }
  }
}

cudaError_t large_build_tables(const LgSched& G, float2* thi, float2* thi_lo, float2* tlo,
                               float2* tlo_lo, float2* sinff, float2* rcpff, cudaStream_t st) {
  const int nhi = (G.S.Nc + G.B - 1) / G.B;
  int N = nhi > G.B ? nhi : G.B;
  if (G.S.n / 2 + 1 > N) N = G.S.n / 2 + 1;
  lg_table_kernel<<<(N + 255) / 256, 256, 0, st>>>(G, thi, thi_lo, tlo, tlo_lo, sinff, rcpff);
  return cudaGetLastError();
}

// ------------------------------------------------------------ launch

size_t large_level_smem(const LgSched& G, int level, bool ff) {
  const int R = level == 1 ? G.R1 : G.R2;
  const FftSched& SR = level == 1 ? G.S1 : G.S2;
  const int TJ = ff ? (level == 1 ? G.TJF1 : G.TJF2) : (level == 1 ? G.TJ1 : G.TJ2);
  size_t b = (size_t)TJ * R * (ff ? 16 : 8);
  if (!ff) b += (size_t)SR.tw_entries * sizeof(float2);
  return b;
}

#define FIF_LG_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

template <class Cx, bool INV, int LV>
static cudaError_t launch_level(const LgSched& G, const LgSig* d_sigs, int nsig, cudaStream_t st) {
  constexpr bool FF = sizeof(Cx) == 16;
  const FftSched& SR = LV == 1 ? G.S1 : G.S2;
  const int TJ = FF ? (LV == 1 ? G.TJF1 : G.TJF2) : (LV == 1 ? G.TJ1 : G.TJ2);
  const int R = LV == 1 ? G.R1 : G.R2;
  const int tiles = (G.S.Nc / R) / TJ;
  const int threads = ((TJ * SR.T + 31) / 32) * 32;
  const size_t smem = large_level_smem(G, LV, FF);
  const dim3 grid(tiles, nsig);
  switch (SR.E) {
#define FIF_CASE(e)                                                   \
  case e:                                                             \
    lg_level<Cx, INV, e, LV><<<grid, threads, smem, st>>>(d_sigs, G); \
    break;
    FIF_LG_E_LIST(FIF_CASE)
#undef FIF_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class Cx, bool INV, int LV>
static cudaError_t level_attr(const LgSched& G, int smem) {
  const FftSched& SR = LV == 1 ? G.S1 : G.S2;
  switch (SR.E) {
#define FIF_CASE(e) \
  case e:           \
    return cudaFuncSetAttribute(lg_level<Cx, INV, e, LV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    FIF_LG_E_LIST(FIF_CASE)
#undef FIF_CASE
  }
  return cudaErrorInvalidValue;
}

// Allow the level kernels this length uses the device's whole opt-in shared
// memory (the instantiations are shared by lengths with other needs); call
// before any stream capture.
cudaError_t large_set_attrs(const LgSched& G) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = level_attr<ffc, false, 1>(G, optin);
  if (e == cudaSuccess) e = level_attr<ffc, false, 2>(G, optin);
  if (e == cudaSuccess) e = level_attr<float2, true, 1>(G, optin);
  if (e == cudaSuccess) e = level_attr<float2, true, 2>(G, optin);
  return e;
}

cudaError_t large_run(const LgSched& G, const LgSig* d_sigs, int nsig, const MethodParams& mp,
                      const float* signals, const Outputs& out, cudaStream_t st) {
  const int pts = G.S.odd ? G.S.n : G.S.Nc;
  const int bx_pts = (pts + 255) / 256 < 1024 ? (pts + 255) / 256 : 1024;
  const int bx_bins = (G.S.P + 255) / 256 < 1024 ? (G.S.P + 255) / 256 : 1024;
  const int nc = G.S.Nc;
  const int bx_half = (nc / 2 + 256) / 256 < 1024 ? (nc / 2 + 256) / 256 : 1024;
  const int bx_split = G.S.odd ? bx_bins : bx_half;
  lg_pack<<<dim3(bx_pts, nsig), 256, 0, st>>>(d_sigs, G, signals);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_level<ffc, false, 1>(G, d_sigs, nsig, st);
  if (e == cudaSuccess) e = launch_level<ffc, false, 2>(G, d_sigs, nsig, st);
  if (e == cudaSuccess) {
    lg_split_fwd<<<dim3(bx_split, nsig), 256, 0, st>>>(d_sigs, G);
    e = cudaGetLastError();
  }
  for (int it = 0; e == cudaSuccess && it <= mp.max_imfs; it++) {
    lg_ctl<<<nsig, 512, 0, st>>>(d_sigs, G, mp, it, signals, out);
    lg_row<<<dim3(bx_bins, nsig), 256, 0, st>>>(d_sigs, G);
    lg_select<<<nsig, 512, 0, st>>>(d_sigs, G, mp);
    lg_multiply<<<dim3(bx_bins, nsig), 256, 0, st>>>(d_sigs, G);
    lg_presplit<<<dim3(bx_split, nsig), 256, 0, st>>>(d_sigs, G);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_level<float2, true, 1>(G, d_sigs, nsig, st);
    if (e == cudaSuccess) e = launch_level<float2, true, 2>(G, d_sigs, nsig, st);
    if (e == cudaSuccess) {
      lg_epilogue<<<dim3(bx_pts, nsig), 256, 0, st>>>(d_sigs, G, out.imfs);
      e = cudaGetLastError();
    }
  }
  return e;
}

}  // namespace fif
