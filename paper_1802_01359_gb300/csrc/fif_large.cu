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
//   extrema   (first iteration only) extrema and zero-crossing count of the
//             input over the whole grid; later counts come from the epilogue
//   ctl       one thread per signal: bookkeeping of the last IMF, outer-loop
//             test (Algorithm 2)
//   row       window eigenvalues {log2(1-w_hat_k), w_hat_k} for this L, in
//             float-float from sine and reciprocal-sine tables; on a stop,
//             the remainder row instead
//   sel32/64  m by eq. SD: rounds of an 8-way search over j, each an FP32
//             screen of SD_j at 8 values of j over the whole grid, then a
//             binary64 pass for the values the screen cannot decide; the last
//             CTA to finish a pass merges the partials and takes the decision
//             (classes of 8 or more signals: one CTA per signal, bisection)
//   multiply  IMF_hat = (1-w_hat)^m r_hat, r_hat <- (1 - (1-w_hat)^m) r_hat,
//             fused with the inverse real-transform split
//   level 1/2 inverse complex FFT
//   epilogue  IMF row = C2R / n, r <- r - IMF (into the other remainder
//             buffer), fused with the extrema count of the new remainder
#include <map>

#include "fif_device.cuh"
#include "fif_tc.cuh"

namespace fif {

// State words of one signal (zeroed before each run).
enum {
  LG_K = 0, LG_FLAGS, LG_DONE, LG_L, LG_M, LG_IFLAGS, LG_SMAX, LG_BAD, LG_IMAX,
  LG_EXT, LG_ZC, LG_TIE, LG_RMAX,         // extrema count of the remainder (atomics)
  LG_LO, LG_HI, LG_STAT, LG_AMB, LG_CNT,  // m search: bracket, statuses, arrivals
  LG_PTIE, LG_PAD,                        // spectral peak: tie flag
  LG_PK, LG_PK_HI,                        // spectral peak key (8-byte aligned word pair)
  LG_KDC, LG_SPAD,                        // shape window: last bin next to DC to redo
  LG_P0, LG_P0_HI,                        // shape window: H_0^2 (binary64, 8-byte aligned)
  LG_ROWOK,                               // 1: this iteration's L is the last one's, its row stands
  LG_NWORDS
};
static_assert(LG_PK % 2 == 0, "64-bit atomics on the peak key");
static_assert(LG_NWORDS <= kLgStateWords, "state words");
static_assert(LG_P0 % 2 == 0, "binary64 H_0^2 in two aligned words");

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
  const int a = m >> G.Bs, b = m & (G.B - 1);
  return cmul(__ldg(&G.thi[a]), __ldg(&G.tlo[b]));
}
template <>
__device__ __forceinline__ float2 inter_twiddle<float2, true>(const LgSched& G, int m) {
  return cconj(inter_twiddle<float2, false>(G, m));
}
template <>
__device__ __forceinline__ ffc inter_twiddle<ffc, false>(const LgSched& G, int m) {
  const int a = m >> G.Bs, b = m & (G.B - 1);
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

// The remainder of iteration it (buffers alternate: the epilogue of iteration
// it reads one and writes the other).
__device__ __forceinline__ float* rem_buf(const LgSig& sg, int it) { return (it & 1) ? sg.rem2 : sg.rem; }

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
// SWZ (levels with S.swz set): columns kLgColPad points apart beyond R
// (the transposed tile stores of adjacent columns meet different banks), each
// in the swizzled layout of S.swz (work_slot).
template <class Cx, bool INV, int E, int LV, bool TC = false, bool SWZ = false>
__global__ void __launch_bounds__(512, sizeof(Cx) == 8 ? 2 : 1) lg_level(const LgSig* __restrict__ sigs, LgSched G) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LgSig sg = sigs[blockIdx.y];
  // (both zero during the input's forward transform; later the forward levels
  // transform a shape window's h, which an unchanged L does not need again)
  if (sg.st[LG_DONE] || (!INV && sg.st[LG_ROWOK])) return;
  constexpr bool FF = sizeof(Cx) == 16;
  const FftSched& SR = FF ? (LV == 1 ? G.F1 : G.F2) : (LV == 1 ? G.S1 : G.S2);
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
  const int tile = TJ * R;  // at most E elements per thread (nt >= TJ R / E)
  const int Rp = SWZ ? R + kLgColPad : R;
  auto cslot = [&](int g, int r) { return g * Rp + (SWZ ? work_slot(r, SR.swz) : r); };
  // element f = tid + u nt of the tile is row r = f / TJ of column g = f % TJ;
  // when TJ divides nt, r = r0 + u nt / TJ and g = g0 (no division per element)
  const bool tj_div = nt % TJ == 0;
  const int r0 = tid / TJ, g0 = tid - r0 * TJ, rstep = nt / TJ;
  auto row_col = [&](int u, int f, int& r, int& g) {
    if (tj_div) {
      r = r0 + u * rstep;
      g = g0;
    } else {
      r = f / TJ;
      g = f - r * TJ;
    }
  };
  {
    // all of this thread's loads in flight together, then the transposed
    // stores to shared memory
    Cx v[E];
#pragma unroll
    for (int u = 0; u < E; u++) {
      const int f = tid + u * nt;
      if (f < tile) {
        int r, g;
        row_col(u, f, r, g);
        v[u] = in[j0 + g + r * stride_in];
      }
    }
#pragma unroll
    for (int u = 0; u < E; u++) {
      const int f = tid + u * nt;
      if (f < tile) {
        int r, g;
        row_col(u, f, r, g);
        if (LV == 2) v[u] = cmul(v[u], inter_twiddle<Cx, INV>(G, r * (j0 + g)));
        buf[cslot(g, r)] = v[u];
      }
    }
  }
  float2* q = nullptr;
  if constexpr (!FF) {
    // the folded table in shared memory, unless the schedule has a per-pass table
    if (!SR.ptw) {
      q = reinterpret_cast<float2*>(smem + (size_t)TJ * Rp * sizeof(Cx));
      for (int u = tid; u < SR.tw_entries; u += nt) {
        const float2 w = __ldg(&SR.tw[u]);
        q[tw_slot(u)] = make_float2(w.x, -w.y);
      }
    }
  }
  __syncthreads();
  const int T = SR.T, g = tid / T;
  const int lt = g < TJ ? tid - g * T : T;  // T: inactive in the sub-FFT
  Cx* mine = buf + (size_t)(g < TJ ? g : 0) * Rp;
  if constexpr (FF) {
    fft_inplace<Cx, INV, E, SWZ>(mine, SR, SR, lt);
  } else {
    const TwSrc ts{q, SR.tw, SR.n, SR.tw_fold, SR.ptw};
    if constexpr (TC)
      fft_inplace_tc<INV, SWZ>(reinterpret_cast<float2*>(mine), SR, ts, lt);
    else
      fft_inplace<Cx, INV, E, SWZ>(mine, SR, ts, lt);
  }
  if (LV == 1) {
    // column j0 + gg, row r goes to (j0 + gg) R + r = j0 R + f
    const bool rp2 = (R & (R - 1)) == 0;
    const int rs = __ffs(R) - 1;
#pragma unroll
    for (int u = 0; u < E; u++) {
      const int f = tid + u * nt;
      if (f < tile) {
        const int gg = TJ == 1 ? 0 : rp2 ? f >> rs : f / R, r = f - gg * R;
        out[(size_t)j0 * R + f] = buf[cslot(gg, r)];
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < E; u++) {
      const int f = tid + u * nt;
      if (f < tile) {
        int r, gg;
        row_col(u, f, r, gg);
        out[j0 + gg + r * G.R1] = buf[cslot(gg, r)];
      }
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

// Extrema count, zero crossings, tie test and max |r| of the remainder (same
// definitions as count_extrema), accumulated over the grid into the state.
__global__ void lg_extrema(const LgSig* __restrict__ sigs, LgSched G) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.y];
  int* st = sg.st;
  if (st[LG_DONE] || st[LG_BAD]) return;
  const float tau = tie_tau(__int_as_float(st[LG_SMAX]));
  const float* rem = sg.rem;
  const int n = G.S.n;
  int ext = 0, zc = 0, tie = 0, step;
  float rmax = 0.f;
  for (int i = first_signal_point(step); i < n; i += step) {
    const int im1 = i == 0 ? n - 1 : i - 1;
    const int ip1 = i + 1 == n ? 0 : i + 1;
    const int ip2 = ip1 + 1 == n ? 0 : ip1 + 1;
    const float a = rem[im1], b = rem[i], c = rem[ip1], d = rem[ip2];
    const float dm = b - a, d0 = c - b, dp = d - c;
    ext += (dm > 0.f && d0 < 0.f) || (dm < 0.f && d0 > 0.f);
    zc += (b > 0.f && c < 0.f) || (b < 0.f && c > 0.f);
    tie |= diff_tie(dm, d0, dp, tau);
    rmax = fmaxf(rmax, fabsf(b));
  }
  tie = __syncthreads_or(tie);
  float fe = (float)ext, fz = (float)zc;  // exact: a CTA counts far fewer than 2^24
  block_reduce2(fe, fz, OpAdd(), 0.f, &red);
  float dummy = 0.f;
  block_reduce2(rmax, dummy, OpMax(), 0.f, &red);
  if (threadIdx.x == 0) {
    atomicAdd(&st[LG_EXT], (int)fe);
    atomicAdd(&st[LG_ZC], (int)fz);
    if (tie) atomicOr(&st[LG_TIE], 1);
    atomicMax(&st[LG_RMAX], __float_as_int(rmax));
  }
}

// Spectral peak of the remainder over the grid (FIF_PEAK_MASK): the largest
// key (magnitude bits above the complemented index, as spectral_peak) by a
// 64-bit atomic max, then whether another bin lies within 1e-5 of it.
__global__ void lg_peak(const LgSig* __restrict__ sigs, LgSched G) {
  __shared__ unsigned long long wmax[32];
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  unsigned long long best = 0ull;
  int step;
  for (int k = first_signal_point(step); k < G.S.P; k += step) {
    if (k == 0) continue;
    const float2 z = sg.spec[k];
    const unsigned long long key = peak_key(fmaf(z.x, z.x, z.y * z.y), k);
    best = key > best ? key : best;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wmax[wid] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) best = wmax[w] > best ? wmax[w] : best;
    atomicMax(reinterpret_cast<unsigned long long*>(&sg.st[LG_PK]), best);
  }
}

__global__ void lg_peak_tie(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  const unsigned long long key = *reinterpret_cast<const unsigned long long*>(&sg.st[LG_PK]);
  const int kp = key ? (int)(0xffffffffu - (unsigned)(key & 0xffffffffull)) : 0;
  const float vmax = __uint_as_float((unsigned)(key >> 32));
  int tie = 0, step;
  for (int k = first_signal_point(step); k < G.S.P; k += step) {
    if (k == 0) continue;
    const float2 z = sg.spec[k];
    tie |= k != kp && fmaf(z.x, z.x, z.y * z.y) >= vmax * (1.f - 1e-5f) && vmax > 0.f;
  }
  tie = __syncthreads_or(tie);
  if (tie && threadIdx.x == 0) atomicOr(&sg.st[LG_PTIE], 1);
}

// Bookkeeping of the IMF extracted in the previous iteration and the outer
// loop test of Algorithm 2 (one thread per signal).  On a stop the remainder
// row is written by lg_row; st[LG_DONE] records the iteration + 1.
__global__ void lg_ctl(const LgSig* __restrict__ sigs, LgSched G, MethodParams mp, int it,
                       const float* __restrict__ signals, Outputs o) {
  const LgSig sg = sigs[blockIdx.x];
  const LgIO io = lg_io(sg, signals, o, mp.max_imfs);
  int* st = sg.st;
  if (st[LG_DONE]) return;
  if (it == 0 && st[LG_BAD]) {
    io.n_imfs[0] = 0;
    io.status[0] = FIF_STOP_NONFINITE;
    if (io.diag) io.diag[0] = fif_imf_diag{0, 0, 0, 0.f};
    st[LG_DONE] = it + 1;
    return;
  }
  const int n = G.S.n;
  ExtremaInfo e;
  e.k = st[LG_EXT];
  e.zc = st[LG_ZC];
  e.tie = st[LG_TIE];
  e.rmax = __int_as_float(st[LG_RMAX]);
  st[LG_EXT] = 0;
  st[LG_ZC] = 0;
  st[LG_TIE] = 0;
  st[LG_RMAX] = 0;
  int K = st[LG_K];
  int flags = st[LG_FLAGS];
  if (it > 0) {  // the IMF extracted in the previous iteration
    const int iflags = st[LG_IFLAGS];
    io.m[K] = st[LG_M];
    if (!mp.force_L) io.mask_len[K] = st[LG_L];
    if (io.diag) {
      io.diag[K].flags = iflags;
      io.diag[K].inf_norm = __int_as_float(st[LG_IMAX]);
    }
    flags |= iflags;
    K++;
  } else {
    e.tie = 0;  // the input itself is exact on both sides
  }
  int L = 0, iflags = e.tie ? FIF_FLAG_EXTREMA_TIE : 0;
  int peak = 0;
  if (mp.peak_mask) {
    const unsigned long long key = *reinterpret_cast<const unsigned long long*>(&st[LG_PK]);
    peak = key ? (int)(0xffffffffu - (unsigned)(key & 0xffffffffull)) : 0;
    if (st[LG_PTIE]) iflags |= FIF_FLAG_EXTREMA_TIE;
    st[LG_PK] = 0;
    st[LG_PK_HI] = 0;
    st[LG_PTIE] = 0;
  }
  const int reason = outer_test(e.k, K, n, mp, io.mask_len, L, iflags, peak);
  if (io.diag) {
    io.diag[K].k_extrema = e.k;
    io.diag[K].zero_crossings = e.zc;
  }
  st[LG_K] = K;
  if (reason) {
    flags |= iflags & FIF_FLAG_EXTREMA_TIE;
    io.n_imfs[0] = K;
    io.status[0] = reason | flags;
    if (io.diag) {
      io.diag[K].flags = iflags & FIF_FLAG_EXTREMA_TIE;
      io.diag[K].inf_norm = e.rmax;
    }
    st[LG_FLAGS] = flags;
    st[LG_DONE] = it + 1;
    return;
  }
  st[LG_FLAGS] = flags;
  st[LG_ROWOK] = it > 0 && L == st[LG_L];  // the row of the last iteration's L is still in place
  st[LG_L] = L;
  st[LG_IFLAGS] = iflags;
  st[LG_IMAX] = 0;
  st[LG_LO] = 0;
  st[LG_HI] = mp.max_inner + 1;  // no j tested below delta yet
  st[LG_M] = mp.max_inner;
  st[LG_AMB] = 0;
  st[LG_STAT] = 0;
  st[LG_CNT] = 0;
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
// A signal that stopped in this iteration instead gets its remainder row
// (a NaN input is its own remainder: lg_pack copied it).
__global__ void lg_row(const LgSig* __restrict__ sigs, LgSched G, int it, float* __restrict__ imfs) {
  const LgSig sg = sigs[blockIdx.y];
  const int n = G.S.n;
  int step;
  const int done = sg.st[LG_DONE];
  if (done) {
    if (done == it + 1) {
      float* orow = imfs + sg.out_off + (size_t)sg.st[LG_K] * n;
      const float* r = rem_buf(sg, it);
      for (int i = first_signal_point(step); i < n; i += step) orow[i] = r[i];
    }
    return;
  }
  if (G.shape || sg.st[LG_ROWOK]) return;  // shape rows: the kernels below; same L: kept
  const int L = sg.st[LG_L];
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

// ------------------------------------------------- shape-generated window
// For a shape window each outer iteration builds the row of its own L: the
// filter h (h_i = g((i + 1/2)/L), i < L) goes through the forward float-float
// levels of the input transform (za/zb are free after it), lg_split_shape
// leaves |H_k|^2 in the signal's binary64 row, lg_shape_row turns it into
// w_hat_k = |H_k|^2 / H_0^2 (and the FP32 row), and lg_shape_dc redoes the
// bins next to DC, where 1 - w_hat_k < 2^-12, with shape_om_direct.

__global__ void lg_pack_shape(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE] || sg.st[LG_ROWOK]) return;
  const int L = sg.st[LG_L], Nc = G.S.Nc;
  ffc* za = reinterpret_cast<ffc*>(sg.za);
  int step;
  for (int t = first_signal_point(step); t < Nc; t += step) {
    if (!G.S.odd) {
      const double a = 2 * t < L ? shape_tap(G.shape, G.shape_len, L, 2 * t) : 0.0;
      const double b = 2 * t + 1 < L ? shape_tap(G.shape, G.shape_len, L, 2 * t + 1) : 0.0;
      za[t] = ffc{ff_from_double(a), ff_from_double(b)};
    } else {
      const double a = t < L ? shape_tap(G.shape, G.shape_len, L, t) : 0.0;
      za[t] = ffc{ff_from_double(a), ff{0.f, 0.f}};
    }
  }
}

__device__ __forceinline__ double ffc_power(const ffc& x) {
  const double re = ff_to_double(x.re), im = ff_to_double(x.im);
  return re * re + im * im;
}

// |H_k|^2 into om64 (the split of lg_split_fwd, kept in float-float); H_0^2
// into the state, and the DC-bin marker reset.
__global__ void lg_split_shape(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE] || sg.st[LG_ROWOK]) return;
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
      const double pk = ffc_power(cadd(e, wo));
      sg.om64[k] = pk;
      sg.om64[Nc - k] = ffc_power(csub(e, wo));
      if (k == 0) {
        *reinterpret_cast<double*>(&sg.st[LG_P0]) = pk;
        sg.st[LG_KDC] = 0;
      }
    }
  } else {
    for (int k = first_signal_point(step); k < G.S.P; k += step) {
      const double pk = ffc_power(za[k]);
      sg.om64[k] = pk;
      if (k == 0) {
        *reinterpret_cast<double*>(&sg.st[LG_P0]) = pk;
        sg.st[LG_KDC] = 0;
      }
    }
  }
}

__global__ void lg_shape_row(const LgSig* __restrict__ sigs, LgSched G) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE] || sg.st[LG_ROWOK]) return;
  const double p0 = *reinterpret_cast<const double*>(&sg.st[LG_P0]);
  int kdc = 0, step;
  for (int k = first_signal_point(step); k < G.S.P; k += step) {
    if (k == 0) {
      sg.row[0] = make_float2(-INFINITY, 1.f);
      sg.om64[0] = 0.0;
      continue;
    }
    double w = sg.om64[k] / p0;
    w = w > 1.0 ? 1.0 : w;
    const double om = 1.0 - w;
    sg.row[k] = make_float2((float)(log1p(-w) * 1.4426950408889634), (float)w);
    sg.om64[k] = om;
    if (om < kShapeDirectBelow) kdc = k;
  }
  kdc = warp_reduce(kdc, OpMax());
  if ((threadIdx.x & 31) == 0 && kdc > 0) atomicMax(&sg.st[LG_KDC], kdc);
}

// Bins 1..kdc again, one warp per bin (kShapeDcBlocks CTAs a signal).
constexpr int kShapeDcBlocks = 16;
__global__ void __launch_bounds__(256) lg_shape_dc(const LgSig* __restrict__ sigs, LgSched G) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE] || sg.st[LG_ROWOK]) return;
  const int kdc = sg.st[LG_KDC];
  if (kdc == 0) return;
  const int L = sg.st[LG_L], n = G.S.n;
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const double h = shape_tap(G.shape, G.shape_len, L, i);
    s0 += h;
    s1 += h * (double)i;
  }
  block_reduce2(s0, s1, OpAdd(), 0.0, &red);
  const double inv = 1.0 / s0, c = s1 / s0;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = 1 + blockIdx.x * nw + (threadIdx.x >> 5); k <= kdc; k += gridDim.x * nw) {
    const double om = shape_om_direct(G.shape, G.shape_len, L, n, k, c, inv);
    if (lane == 0) {
      sg.row[k] = make_float2((float)log2(om), (float)(1.0 - om));
      sg.om64[k] = om;
    }
  }
}

// ------------------------------------------------------------ m search

// Candidates of round `round` of the search for m = the first j in
// [1, max_inner] with SD_j < delta (eq. SD, Sec. 4).  Round 0 tests
// max_inner alone (which decides m = max_inner when SD_max_inner >= delta,
// the common case), or every j when max_inner <= kSelCand; a later round
// tests the j strictly inside the bracket (lo, hi) left by the one before:
// all of them if there are at most kSelCand, else kSelCand evenly spaced
// ones.  Candidates are strictly increasing.
__host__ __device__ __forceinline__ int sel_count(int lo, int hi, int jmax, int round) {
  if (round == 0) return jmax <= kSelCand ? jmax : 1;
  const int u = hi - lo - 1;
  return u <= 0 ? 0 : (u < kSelCand ? u : kSelCand);
}
__host__ __device__ __forceinline__ int sel_cand(int lo, int hi, int jmax, int round, int i) {
  if (round == 0) return jmax <= kSelCand ? i + 1 : jmax;
  const int u = hi - lo - 1;
  if (u <= kSelCand) return lo + 1 + i;
  return lo + (int)(((long long)(i + 1) * (u + 1) + kSelCand) / (kSelCand + 1));
}

// Rounds after which every bracket is closed, from the gaps each round can
// leave (the search runs this many rounds; a closed bracket makes the
// remaining ones return at once).  Only the gap sizes that occur are visited.
static int sel_rounds_after(int u, int jmax, std::map<int, int>& memo) {
  if (u <= 0) return 0;
  auto f = memo.find(u);
  if (f != memo.end()) return f->second;
  const int c = sel_count(0, u + 1, jmax, 1);
  int prev = 0, w = 0;
  for (int i = 0; i <= c; i++) {
    const int j = i < c ? sel_cand(0, u + 1, jmax, 1, i) : u + 1;
    const int r = sel_rounds_after(j - prev - 1, jmax, memo);
    if (r > w) w = r;
    prev = j;
  }
  memo[u] = 1 + w;
  return 1 + w;
}

int large_sel_rounds(int jmax) {
  // round 0 leaves (0, jmax) open (max_inner tested alone) or closes it
  std::map<int, int> memo;
  return 1 + (jmax <= kSelCand ? 0 : sel_rounds_after(jmax - 1, jmax, memo));
}

enum { SEL_F = 0, SEL_T = 1, SEL_AMB = 2 };  // SD_j >= delta, SD_j < delta, undecided

struct SelStep {
  int lo, hi, amb;
};

// New bracket from the statuses of this round's candidates: hi = the first
// candidate below delta, lo = the last candidate at or above delta before it.
// Undecided candidates between them (and, in round 0, an undecided max_inner,
// which alone decides m = max_inner when SD_max_inner >= delta) are returned
// in amb for the binary64 pass.
__device__ SelStep sel_update(int lo, int hi, int jmax, int round, unsigned stat) {
  SelStep r{lo, hi, 0};
  const int c = sel_count(lo, hi, jmax, round);
  if (round == 0) {
    const unsigned s = (stat >> (2 * (c - 1))) & 3u;
    if (s == SEL_F) return SelStep{jmax, jmax + 1, 0};
    if (s == SEL_AMB) r.amb |= 1 << (c - 1);
  }
  int iT = c;
  for (int i = 0; i < c; i++)
    if (((stat >> (2 * i)) & 3u) == SEL_T) {
      iT = i;
      break;
    }
  if (iT < c) r.hi = sel_cand(lo, hi, jmax, round, iT);
  for (int i = 0; i < iT; i++)
    if (((stat >> (2 * i)) & 3u) == SEL_F) r.lo = sel_cand(lo, hi, jmax, round, i);
  for (int i = 0; i < iT; i++) {
    const int j = sel_cand(lo, hi, jmax, round, i);
    if (j > r.lo && ((stat >> (2 * i)) & 3u) == SEL_AMB) r.amb |= 1 << i;
  }
  return r;
}

// Store a decided bracket; a closed one gives m (max_inner when no tested j
// had SD_j < delta).
__device__ void sel_commit(int* st, const SelStep& r, int jmax, int flags) {
  st[LG_LO] = r.lo;
  st[LG_HI] = r.hi;
  st[LG_AMB] = 0;
  if (r.hi - r.lo <= 1) {
    if (r.hi == jmax + 1) {
      st[LG_M] = jmax;
      flags |= FIF_FLAG_MAX_INNER_HIT;
    } else {
      st[LG_M] = r.hi;
    }
  }
  st[LG_IFLAGS] |= flags;
}

// Binary64 one-pass sums of exact_sd's terms relative to 2^M.
struct OnlineD {
  double M, num, den;
};

__device__ __forceinline__ OnlineD online_merge_d(OnlineD a, OnlineD b) {
  if (a.M < b.M) {
    const OnlineD t = a;
    a = b;
    b = t;
  }
  if (b.M == -INFINITY) return a;
  const double s = exp2(b.M - a.M);
  return OnlineD{a.M, b.num * s + a.num, b.den * s + a.den};
}

__device__ __forceinline__ OnlineD warp_merge_d(OnlineD o) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    OnlineD b{__shfl_xor_sync(0xffffffffu, o.M, off), __shfl_xor_sync(0xffffffffu, o.num, off),
              __shfl_xor_sync(0xffffffffu, o.den, off)};
    o = online_merge_d(o, b);
  }
  return o;
}

// Partial of CTA b for candidate i: the FP32 screen's five sums at offset 0,
// the binary64 sums at offset 24.
__device__ __forceinline__ float* part32(const LgSig& sg, int b, int i) {
  return reinterpret_cast<float*>(sg.part + ((size_t)b * kSelCand + i) * kSelPartBytes);
}
__device__ __forceinline__ double* part64(const LgSig& sg, int b, int i) {
  return reinterpret_cast<double*>(sg.part + ((size_t)b * kSelCand + i) * kSelPartBytes + 24);
}
static_assert(kSelPartBytes >= 24 + 3 * 8, "partial record");

__device__ __forceinline__ void store_online(float* p, const Online& o) {
  p[0] = o.M;
  p[1] = o.num;
  p[2] = o.den;
  p[3] = o.anum;
  p[4] = o.aden;
}
__device__ __forceinline__ Online load_online_cg(const float* p) {
  return Online{__ldcg(p), __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3), __ldcg(p + 4)};
}

// True in every thread of the last CTA of this signal to reach this point
// (after its partials are visible); resets the arrival counter.
__device__ __forceinline__ bool last_to_arrive(int* cnt) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(cnt, 1) == (int)gridDim.x - 1;
    if (last) *cnt = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

constexpr int kSelThreads = 256;
constexpr int kSelCtaMinSignals = 8;

// FP32 screen of SD_j for this round's candidates over the grid: per bin the
// term of sd_below (sd_term) for each candidate, accumulated online per
// thread, merged per CTA into sg.part; the last CTA merges the CTAs in index
// order and classifies each candidate against delta with the error band of
// this reduction (screen_margin).  ONE: the round tests max_inner alone (one
// accumulator).  Each thread takes the bins k, k + stride, ... in that order,
// kSdBatch of them per step with their loads issued together.
template <bool ONE>
__global__ void __launch_bounds__(kSelThreads) lg_sel32(const LgSig* __restrict__ sigs, LgSched G,
                                                         MethodParams mp, int round) {
  constexpr int NC = ONE ? 1 : kSelCand;
  __shared__ Online wpart[kSelThreads / 32][kSelCand];
  __shared__ Online fin[kSelCand];
  const LgSig sg = sigs[blockIdx.y];
  int* st = sg.st;
  if (st[LG_DONE]) return;
  const int jmax = mp.max_inner, lo = st[LG_LO], hi = st[LG_HI];
  const int c = sel_count(lo, hi, jmax, round);
  if (c == 0) return;
  if (ONE && c != 1) return;  // (the host launches ONE for such rounds only)
  const FftSched& S = G.S;
  const float sc = spectrum_scale(S.n, __int_as_float(st[LG_SMAX]));
  Online o[NC];
  float e2[NC];
#pragma unroll
  for (int i = 0; i < NC; i++) {
    o[i] = Online{-INFINITY, 0.f, 0.f, 0.f, 0.f};
    e2[i] = i < c ? 2.f * (float)(sel_cand(lo, hi, jmax, round, i) - 1) : 0.f;
  }
  const int stride = gridDim.x * blockDim.x;
  for (int k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < S.P; k0 += kSdBatch * stride) {
    float2 z[kSdBatch], tv[kSdBatch];
#pragma unroll
    for (int u = 0; u < kSdBatch; u++) {
      const int k = k0 + u * stride;
      z[u] = k < S.P ? sg.spec[k] : make_float2(0.f, 0.f);
      tv[u] = k < S.P ? sg.row[k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kSdBatch; u++) {
      if (z[u].x == 0.f && z[u].y == 0.f) continue;  // also bins past the end
      const int k = k0 + u * stride;
      const float re = z[u].x * sc, im = z[u].y * sc;
      const float q = parseval_weight(S, k) * fmaf(re, re, im * im);
      if (!(q > 0.f)) continue;
      float qm, qe;
      q_split(q, qm, qe);
      const float w2 = tv[u].y * tv[u].y;
#pragma unroll
      for (int i = 0; i < NC; i++) {
        if (i < c) {
          const float e = e2[i] == 0.f ? 0.f : e2[i] * tv[u].x;
          if (e != -INFINITY) sd_term(qm, qe, e, w2, o[i]);  // w_hat = 1: no weight for j > 1
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NC; i++) {
    if (i < c) {
      const Online r = warp_merge(o[i]);
      if (lane == 0) wpart[wid][i] = r;
    }
  }
  __syncthreads();
  if (threadIdx.x < c) {
    const int i = threadIdx.x;
    Online r{-INFINITY, 0.f, 0.f, 0.f, 0.f};
    for (int w = 0; w < kSelThreads / 32; w++) r = online_merge(r, wpart[w][i]);
    store_online(part32(sg, blockIdx.x, i), r);
  }
  if (!last_to_arrive(&st[LG_CNT])) return;
  const int nb = gridDim.x;
  for (int i = wid; i < c; i += kSelThreads / 32) {
    Online r{-INFINITY, 0.f, 0.f, 0.f, 0.f};
    for (int b = lane; b < nb; b += 32) r = online_merge(r, load_online_cg(part32(sg, b, i)));
    r = warp_merge(r);
    if (lane == 0) fin[i] = r;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  // chain: bins per thread, then the warps of a CTA and the CTAs per lane of
  // the final merge; levels: two warp trees
  const float chain = (float)((S.P + stride - 1) / stride + kSelThreads / 32 + (nb + 31) / 32);
  const float d2 = mp.delta2;
  unsigned stat = 0;
  for (int i = 0; i < c; i++) {
    const Online& r = fin[i];
    const float ratio = r.num / r.den;
    unsigned s = SEL_AMB;
    if (r.den >= 0.5f && ratio == ratio) {
      const float margin = screen_margin(r, chain, 10.f);
      if (ratio <= d2 * (1.f - margin)) s = SEL_T;
      else if (ratio >= d2 * (1.f + margin)) s = SEL_F;
    }
    stat |= s << (2 * i);
  }
  const SelStep r = sel_update(lo, hi, jmax, round, stat);
  if (r.amb) {
    st[LG_STAT] = (int)stat;
    st[LG_AMB] = r.amb;
  } else {
    sel_commit(st, r, jmax, 0);
  }
}

// Binary64 SD_j (the terms of exact_sd, accumulated online) for the
// candidates the screen left undecided; the last CTA resolves them and
// closes the round.
__global__ void __launch_bounds__(kSelThreads) lg_sel64(const LgSig* __restrict__ sigs, LgSched G,
                                                         MethodParams mp, int round) {
  __shared__ double wpart[kSelThreads / 32][3];
  __shared__ double sd[kSelCand];
  const LgSig sg = sigs[blockIdx.y];
  int* st = sg.st;
  if (st[LG_DONE]) return;
  const int amb = st[LG_AMB];
  if (amb == 0) return;
  const int jmax = mp.max_inner, lo = st[LG_LO], hi = st[LG_HI], L = st[LG_L];
  FftSched S = G.S;
  S.om64 = sg.om64;  // shape window: this signal's binary64 row (stride 0)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int stride = gridDim.x * blockDim.x;
  for (int i = 0; i < kSelCand; i++) {
    if (!((amb >> i) & 1)) continue;
    const int j = sel_cand(lo, hi, jmax, round, i);
    OnlineD o{-INFINITY, 0.0, 0.0};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S.P; k += stride) {
      const float2 z = sg.spec[k];
      const double q = (double)parseval_weight(S, k) * ((double)z.x * z.x + (double)z.y * z.y);
      if (!(q > 0.0)) continue;
      const W64 v = win64(S, L, k);
      const double w = v.w;
      double lw = log2(q);
      if (j > 1) lw += 2.0 * (j - 1) * v.hl;
      if (lw == -INFINITY) continue;
      if (lw > o.M) {
        const double s = exp2(o.M - lw);
        o.num *= s;
        o.den *= s;
        o.M = lw;
      }
      const double t = exp2(lw - o.M);
      o.den += t;
      o.num += t * w * w;
    }
    o = warp_merge_d(o);
    __syncthreads();
    if (lane == 0) {
      wpart[wid][0] = o.M;
      wpart[wid][1] = o.num;
      wpart[wid][2] = o.den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      OnlineD r{-INFINITY, 0.0, 0.0};
      for (int w = 0; w < kSelThreads / 32; w++)
        r = online_merge_d(r, OnlineD{wpart[w][0], wpart[w][1], wpart[w][2]});
      double* d = part64(sg, blockIdx.x, i);
      d[0] = r.M;
      d[1] = r.num;
      d[2] = r.den;
    }
  }
  if (!last_to_arrive(&st[LG_CNT])) return;
  const int nb = gridDim.x;
  for (int i = wid; i < kSelCand; i += kSelThreads / 32) {
    if (!((amb >> i) & 1)) continue;
    OnlineD r{-INFINITY, 0.0, 0.0};
    for (int b = lane; b < nb; b += 32) {
      const double* d = part64(sg, b, i);
      r = online_merge_d(r, OnlineD{__ldcg(d), __ldcg(d + 1), __ldcg(d + 2)});
    }
    r = warp_merge_d(r);
    if (lane == 0) sd[i] = r.den > 0.0 ? sqrt(r.num / r.den) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned stat = (unsigned)st[LG_STAT];
  int flags = FIF_FLAG_FP64_TIEBREAK;
  for (int i = 0; i < kSelCand; i++) {
    if (!((amb >> i) & 1)) continue;
    if (fabs(sd[i] - mp.delta) <= 1e-6 * mp.delta) flags |= FIF_FLAG_NEAR_DELTA_TIE;
    const unsigned s = sd[i] < mp.delta ? SEL_T : SEL_F;
    stat = (stat & ~(3u << (2 * i))) | (s << (2 * i));
  }
  SelStep r = sel_update(lo, hi, jmax, round, stat);
  r.amb = 0;  // every candidate that could move the bracket is now decided
  sel_commit(st, r, jmax, flags);
}

// m by eq. SD with one CTA per signal (bisection over j, select_m_on_row):
// the least work per signal, for classes with enough signals to fill the GPU.
__global__ void __launch_bounds__(512, 1) lg_select_cta(const LgSig* __restrict__ sigs, LgSched G,
                                                        MethodParams mp) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.x];
  int* st = sg.st;
  if (st[LG_DONE]) return;
  const int L = st[LG_L];
  int iflags = st[LG_IFLAGS];
  const float sc = spectrum_scale(G.S.n, __int_as_float(st[LG_SMAX]));
  FftSched S = G.S;
  S.om64 = sg.om64;  // shape window: this signal's binary64 row (stride 0)
  const int m = select_m_on_row(sg.spec, S, sg.row, L, mp, sc, iflags, &red);
  if (threadIdx.x == 0) {
    st[LG_M] = m;
    st[LG_IFLAGS] = iflags;
  }
}

// IMF_hat = (1-w_hat)^m r_hat (eq. One step_algo), r_hat <- (1 - (1-w_hat)^m)
// r_hat, and the inverse real-transform split of IMF_hat (same formulas as
// inverse_real) into work2, in one pass: the thread of k (even n) owns the
// bins k and Nc - k (Nyquist for k = 0), which the split combines.
// TH: the thresholded IMF (gamma > 0).  A separate instance, so that the
// plain one keeps the register count (and occupancy) of a streaming kernel.
template <bool TH>
__global__ void lg_multiply_split(const LgSig* __restrict__ sigs, LgSched G, MethodParams mp) {
  const LgSig sg = sigs[blockIdx.y];
  if (sg.st[LG_DONE]) return;
  const int m = sg.st[LG_M], L = sg.st[LG_L];
  const int Nc = G.S.Nc, n = G.S.n;
  FftSched ST = G.S;  // the threshold's binary64 decisions: this signal's row (shape window)
  ST.om64 = sg.om64;
  int step;
  if (!G.S.odd) {
    for (int k = first_signal_point(step); k <= Nc / 2; k += step) {
      const int kc = Nc - k;
      const float2 zk = sg.spec[k], zc = sg.spec[kc];
      float gk, ok, gc, oc;
      if constexpr (TH) {
        multiplier_th(m, sg.row[k].x, ST, L, k, mp, gk, ok);
        multiplier_th(m, sg.row[kc].x, ST, L, kc, mp, gc, oc);
      } else {
        multiplier(m, sg.row[k].x, gk, ok);
        multiplier(m, sg.row[kc].x, gc, oc);
      }
      const float2 xk = make_float2(gk * zk.x, gk * zk.y);
      const float2 xc = make_float2(gc * zc.x, gc * zc.y);
      sg.spec[k] = make_float2(ok * zk.x, ok * zk.y);
      if (kc != k) sg.spec[kc] = make_float2(oc * zc.x, oc * zc.y);
      const float2 f = make_float2(xk.x + xc.x, xk.y - xc.y);
      const float2 g = make_float2(xk.x - xc.x, xk.y + xc.y);
      const float2 wg = cmul(cconj(__ldg(&G.S.tw[k])), g);
      const float2 iwg = make_float2(-wg.y, wg.x);
      sg.work2[k] = cadd(f, iwg);
      if (k != 0) sg.work2[Nc - k] = cconj(csub(f, iwg));
    }
  } else {
    for (int k = first_signal_point(step); k < G.S.P; k += step) {
      const float2 z = sg.spec[k];
      float g, omg;
      if constexpr (TH)
        multiplier_th(m, sg.row[k].x, ST, L, k, mp, g, omg);
      else
        multiplier(m, sg.row[k].x, g, omg);
      const float2 x = make_float2(g * z.x, g * z.y);
      sg.spec[k] = make_float2(omg * z.x, omg * z.y);
      sg.work2[k] = x;
      if (k != 0) sg.work2[n - k] = cconj(x);
    }
  }
}

// New remainder sample j (0 <= j < n): old remainder minus the IMF sample
// (C2R output / n), recomputed from the inputs for the neighbours a thread
// does not own.
__device__ __forceinline__ float new_rem(const float* ro, const float2* w2, int j, bool odd,
                                         float inv_n) {
  if (odd) return ro[j] - w2[j].x * inv_n;
  const float2 z = w2[j >> 1];
  return ro[j] - ((j & 1) ? z.y : z.x) * inv_n;
}

// Time-domain epilogue of one IMF fused with the extrema count of the new
// remainder (same definitions as count_extrema): IMF row = C2R / n to the
// output, new remainder = old - IMF into the other buffer, and per sample the
// extrema, zero-crossing and tie terms from the new values of its neighbours
// (taken from the old buffer and work2, so no CTA waits for another); CTA
// sums go to the state words by atomics, with max |IMF| and max |r|.
// (at most 32 registers: eight 256-thread CTAs an SM for this streaming kernel)
__global__ void __launch_bounds__(256, 8) lg_epilogue_ext(const LgSig* __restrict__ sigs, LgSched G,
                                                           int it, float* __restrict__ imfs) {
  __shared__ RedScratch red;
  const LgSig sg = sigs[blockIdx.y];
  int* st = sg.st;
  if (st[LG_DONE]) return;
  const int n = G.S.n, K = st[LG_K];
  const bool odd = G.S.odd;
  const float inv_n = 1.f / (float)n;
  const float tau = tie_tau(__int_as_float(st[LG_SMAX]));
  const float* ro = rem_buf(sg, it);
  float* rn = rem_buf(sg, it + 1);
  const float2* w2 = sg.work2;
  float* orow = imfs + sg.out_off + (size_t)K * n;
  float imax = 0.f, rmax = 0.f;
  int ext = 0, zc = 0, tie = 0, step;
  if (!odd) {
    // sample pairs (2t, 2t+1) as float2: the remainder buffers are plan-allocated
    // (8-byte aligned), the IMF row is whenever its offset is even; the neighbours
    // 2t-1, 2t+2, 2t+3 come from the pairs t-1 and t+1 (cyclically), with the same
    // arithmetic as new_rem
    const float2* ro2 = reinterpret_cast<const float2*>(ro);
    float2* rn2 = reinterpret_cast<float2*>(rn);
    const bool vec = (reinterpret_cast<uintptr_t>(orow) & 7) == 0;
    const int Nc = G.S.Nc;
    for (int t = first_signal_point(step); t < Nc; t += step) {
      const int tm = t == 0 ? Nc - 1 : t - 1, tp = t + 1 == Nc ? 0 : t + 1;
      const float2 z = w2[t], zm = w2[tm], zp = w2[tp];
      const float2 q = ro2[t], qm = ro2[tm], qp = ro2[tp];
      const float a = z.x * inv_n, b = z.y * inv_n;
      if (vec) {
        *reinterpret_cast<float2*>(orow + 2 * (size_t)t) = make_float2(a, b);
      } else {
        orow[2 * t] = a;
        orow[2 * t + 1] = b;
      }
      const float r0 = q.x - a, r1 = q.y - b;
      rn2[t] = make_float2(r0, r1);
      imax = fmaxf(imax, fmaxf(fabsf(a), fabsf(b)));
      rmax = fmaxf(rmax, fmaxf(fabsf(r0), fabsf(r1)));
      const float rm1 = qm.y - zm.y * inv_n;
      const float r2 = qp.x - zp.x * inv_n;
      const float r3 = qp.y - zp.y * inv_n;
      pair_terms(rm1, r0, r1, r2, r3, tau, ext, zc, tie);
    }
  } else {
    for (int i = first_signal_point(step); i < n; i += step) {
      const float a = w2[i].x * inv_n;
      orow[i] = a;
      const float b = ro[i] - a;
      rn[i] = b;
      imax = fmaxf(imax, fabsf(a));
      rmax = fmaxf(rmax, fabsf(b));
      const int im1 = i == 0 ? n - 1 : i - 1;
      const int ip1 = i + 1 == n ? 0 : i + 1;
      const int ip2 = ip1 + 1 == n ? 0 : ip1 + 1;
      const float ra = new_rem(ro, w2, im1, true, inv_n), c = new_rem(ro, w2, ip1, true, inv_n);
      const float d = new_rem(ro, w2, ip2, true, inv_n);
      const float dm = b - ra, d0 = c - b, dp = d - c;
      ext += (dm > 0.f && d0 < 0.f) || (dm < 0.f && d0 > 0.f);
      zc += (b > 0.f && c < 0.f) || (b < 0.f && c > 0.f);
      tie |= diff_tie(dm, d0, dp, tau);
    }
  }
  tie = __syncthreads_or(tie);
  float fe = (float)ext, fz = (float)zc;  // exact: a CTA counts far fewer than 2^24
  block_reduce2(fe, fz, OpAdd(), 0.f, &red);
  block_reduce2(imax, rmax, OpMax(), 0.f, &red);
  if (threadIdx.x == 0) {
    atomicAdd(&st[LG_EXT], (int)fe);
    atomicAdd(&st[LG_ZC], (int)fz);
    if (tie) atomicOr(&st[LG_TIE], 1);
    atomicMax(&st[LG_RMAX], __float_as_int(rmax));
    atomicMax(&st[LG_IMAX], __float_as_int(imax));
  }
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
  const FftSched& SR = ff ? (level == 1 ? G.F1 : G.F2) : (level == 1 ? G.S1 : G.S2);
  const int TJ = ff ? (level == 1 ? G.TJF1 : G.TJF2) : (level == 1 ? G.TJ1 : G.TJ2);
  size_t b = (size_t)TJ * (SR.swz ? R + kLgColPad : R) * (ff ? 16 : 8);
  if (!ff && !SR.ptw) b += tw_slots(SR) * sizeof(float2);
  return b;
}

#define FIF_LG_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

template <class Cx, bool INV, int LV>
static cudaError_t launch_level(const LgSched& G, const LgSig* d_sigs, int nsig, cudaStream_t st) {
  constexpr bool FF = sizeof(Cx) == 16;
  const FftSched& SR = FF ? (LV == 1 ? G.F1 : G.F2) : (LV == 1 ? G.S1 : G.S2);
  const int TJ = FF ? (LV == 1 ? G.TJF1 : G.TJF2) : (LV == 1 ? G.TJ1 : G.TJ2);
  const int R = LV == 1 ? G.R1 : G.R2;
  const int tiles = (G.S.Nc / R) / TJ;
  const int threads = ((TJ * SR.T + 31) / 32) * 32;
  const size_t smem = large_level_smem(G, LV, FF);
  const dim3 grid(tiles, nsig);
  if constexpr (!FF && INV) {
    if (LV == 1 ? G.tc1 : G.tc2) {  // split-BF16 tensor-core radix-16 passes (E = 16)
      if (SR.E != 16) return cudaErrorInvalidValue;
      if (SR.swz)
        lg_level<Cx, INV, 16, LV, true, true><<<grid, threads, smem, st>>>(d_sigs, G);
      else
        lg_level<Cx, INV, 16, LV, true><<<grid, threads, smem, st>>>(d_sigs, G);
      return cudaGetLastError();
    }
    if (SR.swz) {  // swizzled columns (E = 8 and 16 schedules only)
      if (SR.E == 8)
        lg_level<Cx, INV, 8, LV, false, true><<<grid, threads, smem, st>>>(d_sigs, G);
      else if (SR.E == 16)
        lg_level<Cx, INV, 16, LV, false, true><<<grid, threads, smem, st>>>(d_sigs, G);
      else
        return cudaErrorInvalidValue;
      return cudaGetLastError();
    }
  }
  if constexpr (FF) {
    if (SR.swz) {  // swizzled columns (the forward levels' E = 8 schedules)
      if (SR.E != 8) return cudaErrorInvalidValue;
      lg_level<Cx, INV, 8, LV, false, true><<<grid, threads, smem, st>>>(d_sigs, G);
      return cudaGetLastError();
    }
  }
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
  const FftSched& SR = sizeof(Cx) == 16 ? (LV == 1 ? G.F1 : G.F2) : (LV == 1 ? G.S1 : G.S2);
  if constexpr (sizeof(Cx) == 8 && INV) {
    if (LV == 1 ? G.tc1 : G.tc2)
      return SR.swz ? cudaFuncSetAttribute(lg_level<Cx, INV, 16, LV, true, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                    : cudaFuncSetAttribute(lg_level<Cx, INV, 16, LV, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (SR.swz) {
      if (SR.E == 8)
        return cudaFuncSetAttribute(lg_level<Cx, INV, 8, LV, false, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (SR.E == 16)
        return cudaFuncSetAttribute(lg_level<Cx, INV, 16, LV, false, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      return cudaErrorInvalidValue;
    }
  }
  if constexpr (sizeof(Cx) == 16) {
    if (SR.swz)
      return SR.E == 8 ? cudaFuncSetAttribute(lg_level<Cx, INV, 8, LV, false, true>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                       : cudaErrorInvalidValue;
  }
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

// The launches of large_run below, counted the same way: pack, two forward
// levels and the split; the input's extrema; then per outer iteration the
// peak pair (peak mode), control, window row, the shape window's six (pack,
// two forward levels, split, row, DC bins), the m search (one CTA kernel, or
// two kernels a round), multiply, two inverse levels and the epilogue.
int large_launches(int nsig, const MethodParams& mp, bool shape) {
  const bool cta_select = nsig >= kSelCtaMinSignals || mp.apriori;
  const int sel = cta_select ? 1 : 2 * large_sel_rounds(mp.max_inner);
  const int per_it = (mp.peak_mask ? 2 : 0) + 2 + sel + 1 + 2 + 1 + (shape ? 6 : 0);
  return 4 + 1 + (mp.max_imfs + 1) * per_it;
}

cudaError_t large_run(const LgSched& G, const LgSig* d_sigs, int nsig, const MethodParams& mp,
                      const float* signals, const Outputs& out, cudaStream_t st) {
  const int pts = G.S.odd ? G.S.n : G.S.Nc;
  const int bx_pts = (pts + 255) / 256 < 1024 ? (pts + 255) / 256 : 1024;
  const int bx_bins = (G.S.P + 255) / 256 < 1024 ? (G.S.P + 255) / 256 : 1024;
  const int nc = G.S.Nc;
  const int bx_half = (nc / 2 + 256) / 256 < 1024 ? (nc / 2 + 256) / 256 : 1024;
  const int bx_split = G.S.odd ? bx_bins : bx_half;
  const int bx_n = (G.S.n + 255) / 256 < 1024 ? (G.S.n + 255) / 256 : 1024;
  const int rounds = large_sel_rounds(mp.max_inner);
  // The grid-wide search does about three times the work of one bisection
  // per signal but spreads one signal over the whole GPU: it pays off for
  // classes of few signals.
  const bool cta_select = nsig >= kSelCtaMinSignals || mp.apriori;  // a-priori m: one CTA
  lg_pack<<<dim3(bx_pts, nsig), 256, 0, st>>>(d_sigs, G, signals);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_level<ffc, false, 1>(G, d_sigs, nsig, st);
  if (e == cudaSuccess) e = launch_level<ffc, false, 2>(G, d_sigs, nsig, st);
  if (e == cudaSuccess) {
    lg_split_fwd<<<dim3(bx_split, nsig), 256, 0, st>>>(d_sigs, G);
    e = cudaGetLastError();
  }
  for (int it = 0; e == cudaSuccess && it <= mp.max_imfs; it++) {
    // the extrema of the input; later iterations count in the epilogue
    if (it == 0) lg_extrema<<<dim3(bx_n, nsig), 256, 0, st>>>(d_sigs, G);
    if (mp.peak_mask) {
      lg_peak<<<dim3(bx_bins, nsig), 256, 0, st>>>(d_sigs, G);
      lg_peak_tie<<<dim3(bx_bins, nsig), 256, 0, st>>>(d_sigs, G);
    }
    lg_ctl<<<nsig, 1, 0, st>>>(d_sigs, G, mp, it, signals, out);
    lg_row<<<dim3(bx_bins, nsig), 256, 0, st>>>(d_sigs, G, it, out.imfs);
    if (G.shape) {
      lg_pack_shape<<<dim3(bx_pts, nsig), 256, 0, st>>>(d_sigs, G);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = launch_level<ffc, false, 1>(G, d_sigs, nsig, st);
      if (e == cudaSuccess) e = launch_level<ffc, false, 2>(G, d_sigs, nsig, st);
      if (e != cudaSuccess) break;
      lg_split_shape<<<dim3(bx_split, nsig), 256, 0, st>>>(d_sigs, G);
      lg_shape_row<<<dim3(bx_bins, nsig), 256, 0, st>>>(d_sigs, G);
      lg_shape_dc<<<dim3(kShapeDcBlocks, nsig), 256, 0, st>>>(d_sigs, G);
    }
    if (cta_select) {
      lg_select_cta<<<nsig, 512, 0, st>>>(d_sigs, G, mp);
    } else {
      for (int r = 0; r < rounds; r++) {
        if (sel_count(0, 0, mp.max_inner, r) == 1 && r == 0)  // max_inner tested alone
          lg_sel32<true><<<dim3(G.sel_blocks, nsig), kSelThreads, 0, st>>>(d_sigs, G, mp, r);
        else
          lg_sel32<false><<<dim3(G.sel_blocks, nsig), kSelThreads, 0, st>>>(d_sigs, G, mp, r);
        lg_sel64<<<dim3(G.sel_blocks, nsig), kSelThreads, 0, st>>>(d_sigs, G, mp, r);
      }
    }
    if (mp.threshold)
      lg_multiply_split<true><<<dim3(bx_split, nsig), 256, 0, st>>>(d_sigs, G, mp);
    else
      lg_multiply_split<false><<<dim3(bx_split, nsig), 256, 0, st>>>(d_sigs, G, mp);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_level<float2, true, 1>(G, d_sigs, nsig, st);
    if (e == cudaSuccess) e = launch_level<float2, true, 2>(G, d_sigs, nsig, st);
    if (e == cudaSuccess) {
      lg_epilogue_ext<<<dim3(bx_pts, nsig), 256, 0, st>>>(d_sigs, G, it, out.imfs);
      e = cudaGetLastError();
    }
  }
  return e;
}

}  // namespace fif
