// Device building blocks of the FIF path: shared-memory Stockham FFTs, the
// m selection of eq. SD through Parseval, the spectral multiplier, and the
// remainder update with the extrema count.  Every function here is called by
// all threads of a CTA (it contains __syncthreads) and works on generic
// pointers, so the fused kernel passes shared memory and the staged kernels
// pass global scratch where they do not stage it.
#pragma once

#include <float.h>
#include <math.h>
#include <stdint.h>

#include "fif_internal.h"

namespace fif {

// ------------------------------------------------------------ complex ops

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 chalf(float2 a) { return make_float2(0.5f * a.x, 0.5f * a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(s * a.x, s * a.y); }

// -i*a for the forward transform, +i*a for the inverse
template <bool INV>
__device__ __forceinline__ float2 rot_i(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// exp(-i theta) * a (forward) or exp(+i theta) * a (inverse), given cos and sin of theta
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a, float c, float s) {
  const float ss = INV ? s : -s;
  return make_float2(c * a.x - ss * a.y, c * a.y + ss * a.x);
}

// ------------------------------------------------- float-float arithmetic
// A value hi + lo held in two floats (|lo| <= ulp(hi)/2), about 48 significant
// bits on the FP32 pipe: Knuth's TwoSum and the FMA form of Dekker's
// TwoProduct, each followed by a fast renormalisation.  The _rn intrinsics
// are never contracted into FMAs, which would break the error-free steps.
struct ff {
  float hi, lo;
};
struct __align__(16) ffc {
  ff re, im;
};

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  return ff{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float hi = __fadd_rn(p, e);
  return ff{hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

__device__ __forceinline__ ffc cadd(ffc a, ffc b) { return ffc{ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ ffc csub(ffc a, ffc b) { return ffc{ff_sub(a.re, b.re), ff_sub(a.im, b.im)}; }
__device__ __forceinline__ ffc cmul(ffc a, ffc w) {
  return ffc{ff_sub(ff_mul(a.re, w.re), ff_mul(a.im, w.im)),
             ff_add(ff_mul(a.re, w.im), ff_mul(a.im, w.re))};
}
__device__ __forceinline__ ffc cconj(ffc a) { return ffc{a.re, ff_neg(a.im)}; }
__device__ __forceinline__ ffc chalf(ffc a) {
  return ffc{ff{0.5f * a.re.hi, 0.5f * a.re.lo}, ff{0.5f * a.im.hi, 0.5f * a.im.lo}};
}
__device__ __forceinline__ ffc cscale(ffc a, ff s) { return ffc{ff_mul(a.re, s), ff_mul(a.im, s)}; }
template <bool INV>
__device__ __forceinline__ ffc rot_i(ffc a) {
  return INV ? ffc{ff_neg(a.im), a.re} : ffc{a.im, ff_neg(a.re)};
}
template <bool INV>
__device__ __forceinline__ ffc rot(ffc a, ff c, ff s) {
  const ff ss = INV ? s : ff_neg(s);
  return ffc{ff_sub(ff_mul(c, a.re), ff_mul(ss, a.im)), ff_add(ff_mul(c, a.im), ff_mul(ss, a.re))};
}

// Butterfly constants for each arithmetic: cos(pi/8), sin(pi/8), sqrt(1/2),
// sin(2 pi/3); float-float pairs are the binary32 value and the rounded rest.
template <class Cx>
struct Kc;
template <>
struct Kc<float2> {
  __device__ static float c16() { return 0.923879532511286756f; }
  __device__ static float s16() { return 0.382683432365089772f; }
  __device__ static float r2() { return 0.707106781186547524f; }
  __device__ static float h3() { return 0.866025403784438647f; }
  // cos and sin of 2 pi m/9, m = 1, 2, 4 (the radix-9 twiddles)
  __device__ static float c91() { return 0.766044443118978035f; }
  __device__ static float s91() { return 0.642787609686539326f; }
  __device__ static float c92() { return 0.173648177666930349f; }
  __device__ static float s92() { return 0.984807753012208059f; }
  __device__ static float c94() { return -0.939692620785908384f; }
  __device__ static float s94() { return 0.342020143325668733f; }
  __device__ static float neg(float a) { return -a; }
};
template <>
struct Kc<ffc> {
  __device__ static ff c16() { return ff{0.9238795042037964f, 2.830748968563057e-08f}; }
  __device__ static ff s16() { return ff{0.3826834261417389f, 6.2233507236442165e-09f}; }
  __device__ static ff r2() { return ff{0.7071067690849304f, 1.2101617485882343e-08f}; }
  __device__ static ff h3() { return ff{0.8660253882408142f, 1.5543625053737742e-08f}; }
  __device__ static ff c91() { return ff{0.7660444378852844f, 5.2336934786012534e-09f}; }
  __device__ static ff s91() { return ff{0.6427876353263855f, -2.5639845802061245e-08f}; }
  __device__ static ff c92() { return ff{0.1736481785774231f, -9.10492736760915e-10f}; }
  __device__ static ff s92() { return ff{0.9848077297210693f, 2.3291137907222037e-08f}; }
  __device__ static ff c94() { return ff{-0.9396926164627075f, -4.323200908373792e-09f}; }
  __device__ static ff s94() { return ff{0.3420201539993286f, -1.0673660177928923e-08f}; }
  __device__ static ff neg(ff a) { return ff_neg(a); }
};

// Twiddle exp(-+2 pi i idx/n) from the plan's table (hi part, and for
// float-float the rounded rest).
template <class Cx, bool INV>
__device__ __forceinline__ Cx load_tw(const FftSched& S, int idx);
template <>
__device__ __forceinline__ float2 load_tw<float2, false>(const FftSched& S, int idx) {
  return __ldg(&S.tw[idx]);
}
template <>
__device__ __forceinline__ float2 load_tw<float2, true>(const FftSched& S, int idx) {
  return cconj(__ldg(&S.tw[idx]));
}
template <>
__device__ __forceinline__ ffc load_tw<ffc, false>(const FftSched& S, int idx) {
  const float2 h = __ldg(&S.tw[idx]), l = __ldg(&S.tw_lo[idx]);
  return ffc{ff{h.x, l.x}, ff{h.y, l.y}};
}
template <>
__device__ __forceinline__ ffc load_tw<ffc, true>(const FftSched& S, int idx) {
  return cconj(load_tw<ffc, false>(S, idx));
}

// ------------------------------------------------------- small DFT kernels

template <class Cx, bool INV>
__device__ __forceinline__ void dft2(Cx* v) {
  const Cx a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <class Cx, bool INV>
__device__ __forceinline__ void dft3(Cx* v) {
  const Cx t1 = cadd(v[1], v[2]);
  const Cx t2 = csub(v[0], chalf(t1));
  const Cx t3 = rot_i<INV>(cscale(csub(v[1], v[2]), Kc<Cx>::h3()));
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, t3);
  v[2] = csub(t2, t3);
}

template <class Cx, bool INV>
__device__ __forceinline__ void dft3r(Cx& a, Cx& b, Cx& c) {
  const Cx t1 = cadd(b, c);
  const Cx t2 = csub(a, chalf(t1));
  const Cx t3 = rot_i<INV>(cscale(csub(b, c), Kc<Cx>::h3()));
  a = cadd(a, t1);
  b = cadd(t2, t3);
  c = csub(t2, t3);
}

// 9 = 3 x 3: DFT3 over x[3 n1 + n2], twiddle w9^(n2 k1), DFT3 over n2; one
// pass of shared-memory traffic where two radix-3 passes took two.
template <class Cx, bool INV>
__device__ __forceinline__ void dft9(Cx* v) {
#pragma unroll
  for (int n2 = 0; n2 < 3; n2++) dft3r<Cx, INV>(v[n2], v[3 + n2], v[6 + n2]);
  // v[3 k1 + n2] now holds Y[n2][k1]
  v[4] = rot<INV>(v[4], Kc<Cx>::c91(), Kc<Cx>::s91());
  v[7] = rot<INV>(v[7], Kc<Cx>::c92(), Kc<Cx>::s92());
  v[5] = rot<INV>(v[5], Kc<Cx>::c92(), Kc<Cx>::s92());
  v[8] = rot<INV>(v[8], Kc<Cx>::c94(), Kc<Cx>::s94());
#pragma unroll
  for (int k1 = 0; k1 < 3; k1++) dft3r<Cx, INV>(v[3 * k1], v[3 * k1 + 1], v[3 * k1 + 2]);
  // v[3 k1 + k2] now holds X[k1 + 3 k2]: transpose the 3 x 3 block
  Cx t;
  t = v[1], v[1] = v[3], v[3] = t;
  t = v[2], v[2] = v[6], v[6] = t;
  t = v[5], v[5] = v[7], v[7] = t;
}

template <class Cx, bool INV>
__device__ __forceinline__ void dft4r(Cx& x0, Cx& x1, Cx& x2, Cx& x3) {
  const Cx t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = rot_i<INV>(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

template <class Cx, bool INV>
__device__ __forceinline__ void dft4(Cx* v) {
  dft4r<Cx, INV>(v[0], v[1], v[2], v[3]);
}

// 8 = 4 x 2: four-point DFTs over the even and odd samples, twiddle, pairs.
template <class Cx, bool INV>
__device__ __forceinline__ void dft8(Cx* v) {
  Cx a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6];
  Cx b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
  dft4r<Cx, INV>(a0, a1, a2, a3);
  dft4r<Cx, INV>(b0, b1, b2, b3);
  const auto c = Kc<Cx>::r2();
  b1 = rot<INV>(b1, c, c);
  b2 = rot_i<INV>(b2);
  b3 = rot<INV>(b3, Kc<Cx>::neg(c), c);
  v[0] = cadd(a0, b0);
  v[4] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[5] = csub(a1, b1);
  v[2] = cadd(a2, b2);
  v[6] = csub(a2, b2);
  v[3] = cadd(a3, b3);
  v[7] = csub(a3, b3);
}

// 16 = 4 x 4: DFT4 over x[4 n1 + n2], twiddle w16^(n2 k1), DFT4 over n2.
template <class Cx, bool INV>
__device__ __forceinline__ void dft16(Cx* v) {
#pragma unroll
  for (int n2 = 0; n2 < 4; n2++) dft4r<Cx, INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // v[4 k1 + n2] now holds Y[n2][k1]
  const auto C1 = Kc<Cx>::c16(), S1 = Kc<Cx>::s16(), C2 = Kc<Cx>::r2();
  v[5] = rot<INV>(v[5], C1, S1);
  v[9] = rot<INV>(v[9], C2, C2);
  v[13] = rot<INV>(v[13], S1, C1);
  v[6] = rot<INV>(v[6], C2, C2);
  v[10] = rot_i<INV>(v[10]);
  v[14] = rot<INV>(v[14], Kc<Cx>::neg(C2), C2);
  v[7] = rot<INV>(v[7], S1, C1);
  v[11] = rot<INV>(v[11], Kc<Cx>::neg(C2), C2);
  v[15] = rot<INV>(v[15], Kc<Cx>::neg(C1), Kc<Cx>::neg(S1));
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++) dft4r<Cx, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // v[4 k1 + k2] now holds X[k1 + 4 k2]: transpose the 4 x 4 block in registers
  Cx t;
  t = v[1], v[1] = v[4], v[4] = t;
  t = v[2], v[2] = v[8], v[8] = t;
  t = v[3], v[3] = v[12], v[12] = t;
  t = v[6], v[6] = v[9], v[9] = t;
  t = v[7], v[7] = v[13], v[13] = t;
  t = v[11], v[11] = v[14], v[14] = t;
}

template <class Cx, bool INV, int R>
__device__ __forceinline__ void butterfly(Cx* v) {
  if (R == 2) dft2<Cx, INV>(v);
  if (R == 3) dft3<Cx, INV>(v);
  if (R == 4) dft4<Cx, INV>(v);
  if (R == 8) dft8<Cx, INV>(v);
  if (R == 16) dft16<Cx, INV>(v);
  if (R == 9) dft9<Cx, INV>(v);
}

// ------------------------------------------------------- Stockham passes

// Where the FP32 passes take their twiddles from: a folded shared-memory
// table Q[u] = (cos 2 pi u/n, sin 2 pi u/n), u = 0 .. n/2^fold (fold 3 uses the
// octant symmetry, 2 the quarter-wave, 1 the half-wave), or the global table.
struct TwSrc {
  const float2* q;   // shared table or nullptr
  const float2* g;   // global table exp(-2 pi i t/n)
  int n;
  int fold;
  const float2* p;   // or the schedule's per-pass table (FftSched::ptw; inverse direction)
};

// Slot of point i in a swizzled transform buffer: i with its low four bits
// XOR-ed by five times its 16-point block index (mask m = 15), or i itself
// (m = 0).  A bijection inside every aligned block of 16 points, so a
// half-warp reading 16 consecutive points still meets every bank pair once,
// while the Stockham stores R or Ns points apart spread over all bank pairs
// instead of meeting in one (up to 16-way conflicts in the first pass).
__device__ __forceinline__ int work_slot(int i, int m) { return i ^ (((i >> 4) * 5) & m); }

// exp(-2 pi i t/n), 0 <= t < n
__device__ __forceinline__ float2 tw_value(const TwSrc& ts, int t) {
  if (!ts.q) return __ldg(&ts.g[t]);
  const int n = ts.n;
  if (ts.fold >= 2) {
    const int quarter = n >> 2;
    const int qd = (t >= quarter) + (t >= 2 * quarter) + (t >= 3 * quarter);
    const int u = t - qd * quarter;
    const bool sw = ts.fold == 3 && u > (n >> 3);
    const float2 v = ts.q[tw_slot(sw ? quarter - u : u)];
    const float c = sw ? v.y : v.x, s = sw ? v.x : v.y;
    // exp(-i (qd pi/2 + phi)) with cos phi = c, sin phi = s
    const float a = (qd & 1) ? s : c, b = (qd & 1) ? c : s;
    return make_float2((qd == 1 || qd == 2) ? -a : a, qd < 2 ? -b : b);
  }
  if (ts.fold == 1) {
    const int half = n >> 1;
    const bool h = t >= half;
    const float2 v = ts.q[tw_slot(h ? t - half : t)];
    return h ? make_float2(-v.x, v.y) : make_float2(v.x, -v.y);
  }
  const float2 v = ts.q[tw_slot(t)];
  return make_float2(v.x, -v.y);
}

template <bool INV>
__device__ __forceinline__ float2 tw_dir(const TwSrc& ts, int t) {
  const float2 w = tw_value(ts, t);
  return INV ? cconj(w) : w;
}

// Multiply v[1..R-1] by w^r, w = exp(-+2 pi i b/n): w, w^2, w^4, w^8 are looked
// up, the other powers are products of at most three of them.
template <bool INV, int R>
__device__ __forceinline__ void apply_twiddles(float2* v, const TwSrc& ts, int b) {
  const float2 w1 = tw_dir<INV>(ts, b);
  if (R == 2) {
    v[1] = cmul(v[1], w1);
    return;
  }
  const float2 w2 = tw_dir<INV>(ts, 2 * b);
  v[1] = cmul(v[1], w1);
  v[2] = cmul(v[2], w2);
  if (R == 3) return;
  const float2 w3 = cmul(w2, w1);
  v[3] = cmul(v[3], w3);
  if (R == 4) return;
  const float2 w4 = tw_dir<INV>(ts, 4 * b);
  v[4] = cmul(v[4], w4);
  v[5] = cmul(v[5], cmul(w4, w1));
  v[6] = cmul(v[6], cmul(w4, w2));
  const float2 w7 = cmul(w4, w3);
  v[7] = cmul(v[7], w7);
  if (R == 8) return;
  const float2 w8 = tw_dir<INV>(ts, 8 * b);
  v[8] = cmul(v[8], w8);
  if (R == 9) return;
  v[9] = cmul(v[9], cmul(w8, w1));
  v[10] = cmul(v[10], cmul(w8, w2));
  v[11] = cmul(v[11], cmul(w8, w3));
  v[12] = cmul(v[12], cmul(w8, w4));
  v[13] = cmul(v[13], cmul(w8, cmul(w4, w1)));
  v[14] = cmul(v[14], cmul(w8, cmul(w4, w2)));
  v[15] = cmul(v[15], cmul(w8, w7));
}

// Multiply v[1..R-1] by the pass's twiddles w^(r k) read from its per-pass
// table: base = table + (Ns - 1) + k, entry r at base[(r - 1) Ns] (each one
// rounded from binary64; the table holds the inverse direction).
template <bool INV, int R>
__device__ __forceinline__ void apply_pass_twiddles(float2* v, const float2* __restrict__ base,
                                                    int Ns) {
  float2 w[R - 1];
#pragma unroll
  for (int r = 1; r < R; r++) w[r - 1] = __ldg(base + (r - 1) * Ns);
#pragma unroll
  for (int r = 1; r < R; r++) v[r] = cmul(v[r], INV ? w[r - 1] : cconj(w[r - 1]));
}

template <bool INV, int R>
__device__ __forceinline__ void apply_twiddles(ffc* v, const FftSched& S, int b) {
#pragma unroll
  for (int r = 1; r < R; r++) v[r] = cmul(v[r], load_tw<ffc, INV>(S, r * b));
}

template <class Cx>
struct TwArg;
template <>
struct TwArg<float2> {
  using type = TwSrc;
};
template <>
struct TwArg<ffc> {
  using type = FftSched;
};

// One radix-R pass of the self-sorting (Stockham) FFT, in place: every thread
// first loads its E/R butterflies (inputs at j + r*Nc/R), the CTA
// synchronises, then each butterfly is twiddled by w_{Ns R}^{r (j mod Ns)},
// transformed, and stored at (j - j mod Ns) R + j mod Ns + r Ns.  SWZ: point
// i lives in slot work_slot(i, S.swz) of buf.
template <class Cx, bool INV, int R, int E, bool SWZ = false>
__device__ __forceinline__ void fft_pass(Cx* buf, const FftSched& S,
                                         const typename TwArg<Cx>::type& tws, int Ns, int tid) {
  auto slot = [&](int i) { return SWZ ? work_slot(i, S.swz) : i; };
  constexpr int NB = E / R;
  const int T = S.T;
  const int stride = S.Nc / R;
  const bool active = tid < T;
  Cx v[E];
  if (active) {
#pragma unroll
    for (int t = 0; t < NB; t++) {
      const int j = tid + t * T;
#pragma unroll
      for (int r = 0; r < R; r++) v[t * R + r] = buf[slot(j + r * stride)];
    }
  }
  __syncthreads();
  if (active) {
    // j mod Ns: a mask when Ns is a power of two (every pass of a 2^a length),
    // else an integer division
    const bool p2 = (Ns & (Ns - 1)) == 0;
#pragma unroll
    for (int t = 0; t < NB; t++) {
      const int j = tid + t * T;
      int k;
      if (p2)
        k = j & (Ns - 1);
      else
        k = j % Ns;
      if constexpr (sizeof(Cx) == sizeof(float2)) {
        if (k != 0) {
          if (tws.p)
            apply_pass_twiddles<INV, R>(&v[t * R], tws.p + (Ns - 1) + k, Ns);
          else
            apply_twiddles<INV, R>(&v[t * R], tws, k * (S.n / (Ns * R)));
        }
      } else {
        if (k != 0) apply_twiddles<INV, R>(&v[t * R], tws, k * (S.n / (Ns * R)));
      }
      butterfly<Cx, INV, R>(&v[t * R]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; r++) buf[slot(base + r * Ns)] = v[t * R + r];
    }
  }
  __syncthreads();
}

// The one pass whose radix is neither the schedule's main radix nor half of
// it (the host emits at most one such pass per transform, and only for
// power-of-two parts that are not sums of those).  Kept out of line so that
// its register needs do not add to the main loop's.
template <class Cx, bool INV, int E, bool SWZ = false>
__device__ __noinline__ void fft_tail_pass(Cx* buf, const FftSched& S,
                                           const typename TwArg<Cx>::type& tws, int Ns, int R,
                                           int tid) {
  if constexpr (E % 16 == 0) {
    if (R == 16) fft_pass<Cx, INV, 16, E, SWZ>(buf, S, tws, Ns, tid);
  }
  if constexpr (E % 8 == 0) {
    if (R == 8) fft_pass<Cx, INV, 8, E, SWZ>(buf, S, tws, Ns, tid);
  }
  if constexpr (E % 4 == 0) {
    if (R == 4) fft_pass<Cx, INV, 4, E, SWZ>(buf, S, tws, Ns, tid);
  }
  if constexpr (E % 2 == 0) {
    if (R == 2) fft_pass<Cx, INV, 2, E, SWZ>(buf, S, tws, Ns, tid);
  }
}

template <int E>
__host__ __device__ constexpr int main_radix() {
  return E % 16 == 0 ? 16 : E % 8 == 0 ? 8 : E % 4 == 0 ? 4 : E % 2 == 0 ? 2 : 3;
}

// Complex FFT of S.Nc points in buf (unnormalised).  Forward: exp(-2 pi i jk/Nc).
// Every radix of the schedule divides E; all but at most one pass use the
// main radix (largest power of two dividing E, at most 16), half of it, or
// radix 3 (inline); the exception runs out of line.
// tid is the thread's index among the S.T threads of this transform (several
// independent transforms may share a CTA); every thread of the CTA calls it.
template <class Cx, bool INV, int E, bool SWZ = false>
__device__ __forceinline__ void fft_inplace(Cx* buf, const FftSched& S,
                                            const typename TwArg<Cx>::type& tws,
                                            int tid = threadIdx.x) {
  constexpr int RM = main_radix<E>();
  int Ns = 1;
#pragma unroll 1
  for (int p = 0; p < S.npass; p++) {
    const int R = S.radix[p];
    if (R == RM) {
      fft_pass<Cx, INV, RM, E, SWZ>(buf, S, tws, Ns, tid);
    } else if (sizeof(Cx) == 8 && RM >= 4 && R == RM / 2) {
      // FP32 transforms (once per IMF) keep the half-radix pass inline; the
      // float-float forward transform (once per signal) calls it out of line
      if constexpr (sizeof(Cx) == 8 && RM >= 4) fft_pass<Cx, INV, RM / 2, E, SWZ>(buf, S, tws, Ns, tid);
    } else if (E % 9 == 0 && R == 9) {
      if constexpr (E % 9 == 0) fft_pass<Cx, INV, 9, E, SWZ>(buf, S, tws, Ns, tid);
    } else if (E % 3 == 0 && R == 3) {
      if constexpr (E % 3 == 0 && RM != 3) fft_pass<Cx, INV, 3, E, SWZ>(buf, S, tws, Ns, tid);
    } else {
      fft_tail_pass<Cx, INV, E, SWZ>(buf, S, tws, Ns, R, tid);
    }
    Ns *= R;
  }
}

// ------------------------------------------------------------ reductions

struct RedScratch {
  double d[96];
};

template <typename T, typename Op>
__device__ __forceinline__ T warp_reduce(T v, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reduction of two values of type T (float or double) with op;
// every thread gets the result.  scratch holds >= 64 doubles.
template <typename T, typename Op>
__device__ __forceinline__ void block_reduce2(T& a, T& b, Op op, T ident, RedScratch* scratch) {
  a = warp_reduce(a, op);
  b = warp_reduce(b, op);
  T* s = reinterpret_cast<T*>(scratch->d);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    s[2 * wid] = a;
    s[2 * wid + 1] = b;
  }
  __syncthreads();
  T x = lane < nw ? s[2 * lane] : ident;
  T y = lane < nw ? s[2 * lane + 1] : ident;
  x = warp_reduce(x, op);
  y = warp_reduce(y, op);
  a = x;
  b = y;
}

struct OpAdd {
  template <typename T>
  __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
};
struct OpMax {
  template <typename T>
  __device__ __forceinline__ T operator()(T a, T b) const { return a > b ? a : b; }
};

// ------------------------------------------------------ real transforms

// Forward real FFT in float-float arithmetic, rounded once per bin.  An FP32
// forward transform leaves round-off of the order 2^-24 ||s|| in every bin;
// the bins an IMF keeps can hold far less energy than s, so that error
// would dominate the IMF.  Every later step errs relative to the IMF itself.
//   x    n real samples (global)
//   zf   float-float work array of Nc complex points (16 Nc bytes); it may
//        overlay rem and the float work array of the caller, but must not
//        overlap spec[0..P) in its first 16 P bytes
//   spec receives the n/2+1 (even n) or (n+1)/2 (odd n) bins, rounded
//   rem  receives x (written after the transform)
// Returns max |x| (every thread), or -1 if x holds a NaN or Inf.
// Out of line: once per signal, and inlined it raised the register need (and
// the spills) of the per-IMF loop of the kernels that call it.
template <int E>
__device__ __noinline__ float forward_real(const float* __restrict__ x, float* rem, ffc* zf, float2* spec,
                              const FftSched& S, RedScratch* red) {
  const int tid = threadIdx.x, nt = blockDim.x, n = S.n;
  float amax = 0.f;
  int bad = 0;
  if (!S.odd) {
    for (int t = tid; t < S.Nc; t += nt) {
      const float a = x[2 * t], b = x[2 * t + 1];
      zf[t] = ffc{ff{a, 0.f}, ff{b, 0.f}};
      amax = fmaxf(amax, fmaxf(fabsf(a), fabsf(b)));
      bad |= !isfinite(a) || !isfinite(b);
    }
  } else {
    for (int t = tid; t < n; t += nt) {
      const float a = x[t];
      zf[t] = ffc{ff{a, 0.f}, ff{0.f, 0.f}};
      amax = fmaxf(amax, fabsf(a));
      bad |= !isfinite(a);
    }
  }
  bad = __syncthreads_or(bad);
  float dummy = 0.f;
  block_reduce2(amax, dummy, OpMax(), 0.f, red);
  if (bad) return -1.f;
  fft_inplace<ffc, false, E>(zf, S, S);
  if (!S.odd) {
    // X_k = E + W^k O, X_{Nc-k} = conj(E - W^k O),
    // E = (Z_k + conj Z_{Nc-k})/2, O = -i (Z_k - conj Z_{Nc-k})/2, W = exp(-2 pi i/n)
    const int Nc = S.Nc;
    for (int k = tid; k <= Nc / 2; k += nt) {
      const ffc zk = zf[k];
      const ffc zc = cconj(zf[k == 0 ? 0 : Nc - k]);
      const ffc e = chalf(cadd(zk, zc));
      const ffc o = rot_i<false>(chalf(csub(zk, zc)));
      const ffc wo = cmul(load_tw<ffc, false>(S, k), o);
      const ffc xk = cadd(e, wo);
      const ffc xc = cconj(csub(e, wo));
      zf[k] = xk;
      if (k == 0)
        spec[Nc] = make_float2(xc.re.hi, xc.im.hi);
      else
        zf[Nc - k] = xc;
    }
    __syncthreads();
    for (int k = tid; k < Nc; k += nt) spec[k] = make_float2(zf[k].re.hi, zf[k].im.hi);
  } else {
    for (int k = tid; k < S.P; k += nt) spec[k] = make_float2(zf[k].re.hi, zf[k].im.hi);
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) rem[i] = x[i];
  __syncthreads();
  return amax;
}

// Inverse real FFT of the bins in work[0..P) (in place); afterwards the time
// sample t is  work[t/2].x or .y (even n)  or  work[t].x (odd n), times n.
template <int E>
__device__ void inverse_real(float2* work, const FftSched& S, const TwSrc& ts) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!S.odd) {
    // Z_k = F + i W^-k G, Z_{Nc-k} = conj(F - i W^-k G),
    // F = X_k + conj X_{Nc-k}, G = X_k - conj X_{Nc-k}
    const int Nc = S.Nc;
    for (int k = tid; k <= Nc / 2; k += nt) {
      const float2 xk = work[k];
      const float2 xc = work[Nc - k];
      const float2 f = make_float2(xk.x + xc.x, xk.y - xc.y);
      const float2 g = make_float2(xk.x - xc.x, xk.y + xc.y);
      const float2 wg = cmul(cconj(tw_value(ts, k)), g);
      const float2 iwg = make_float2(-wg.y, wg.x);
      work[k] = cadd(f, iwg);
      if (k != 0) work[Nc - k] = cconj(csub(f, iwg));
    }
  } else {
    const int n = S.n;
    for (int k = 1 + tid; k < S.P; k += nt) work[n - k] = cconj(work[k]);
  }
  __syncthreads();
  fft_inplace<float2, true, E>(work, S, ts);
}

// The IMF's spectrum, the spectral remainder update and the inverse real FFT
// in one: on entry work[k] = {g_k, 1 - g_k} (select_m_mult) and spec holds
// r_hat.  The first step applies IMF_hat_k = g_k r_hat_k (eq. One step_algo)
// and r_hat_k <- (1 - g_k) r_hat_k (Algorithm 2: s = s - s_m) to the bin pair
// (k, Nc - k) that the inverse real split combines, so the multiplier needs
// no pass of its own; then the complex inverse FFT.  Afterwards the time
// sample t is work[t/2].x or .y (even n) or work[t].x (odd n), times n.
// mult: the multiplier pairs, either work itself (select_m_mult's pass) or a
// row of the plan's table for m = max_inner (global memory).
__device__ __forceinline__ void inverse_real_mult_split(float2* spec, float2* work,
                                                        const float2* mult, const FftSched& S,
                                                        const TwSrc& ts) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!S.odd) {
    const int Nc = S.Nc;
    for (int k = tid; k <= Nc / 2; k += nt) {
      const int kc = Nc - k;
      const float2 gk = mult[k], gc = mult[kc];
      const float2 zk = spec[k], zc = spec[kc];
      const float2 xk = make_float2(gk.x * zk.x, gk.x * zk.y);
      const float2 xc = make_float2(gc.x * zc.x, gc.x * zc.y);
      spec[k] = make_float2(gk.y * zk.x, gk.y * zk.y);
      if (kc != k) spec[kc] = make_float2(gc.y * zc.x, gc.y * zc.y);
      // Z_k = F + i W^-k G, Z_{Nc-k} = conj(F - i W^-k G),
      // F = X_k + conj X_{Nc-k}, G = X_k - conj X_{Nc-k}
      const float2 f = make_float2(xk.x + xc.x, xk.y - xc.y);
      const float2 g = make_float2(xk.x - xc.x, xk.y + xc.y);
      const float2 wg = cmul(cconj(tw_value(ts, k)), g);
      const float2 iwg = make_float2(-wg.y, wg.x);
      work[k] = cadd(f, iwg);
      if (k != 0) work[kc] = cconj(csub(f, iwg));
    }
  } else {
    const int n = S.n;
    for (int k = tid; k < S.P; k += nt) {
      const float2 gk = mult[k], zk = spec[k];
      const float2 x = make_float2(gk.x * zk.x, gk.x * zk.y);
      spec[k] = make_float2(gk.y * zk.x, gk.y * zk.y);
      work[k] = x;
      if (k != 0) work[n - k] = cconj(x);
    }
  }
  __syncthreads();
}

template <int E>
__device__ void inverse_real_mult(float2* spec, float2* work, const float2* mult, const FftSched& S,
                                  const TwSrc& ts) {
  inverse_real_mult_split(spec, work, mult, S, ts);
  fft_inplace<float2, true, E>(work, S, ts);
}

// ---------------------------------------------------------- window table

__device__ __forceinline__ const float2* wrow(const FftSched& S, int L) {
  return S.wtab + (size_t)(L - 1) * (size_t)S.P;
}

__device__ __forceinline__ float parseval_weight(const FftSched& S, int k) {
  return (k == 0 || (!S.odd && 2 * k == S.n)) ? 1.f : 2.f;
}

// w_hat_k in binary64 from the sine table (exact integer argument reduction).
__device__ __forceinline__ double what64(const FftSched& S, int L, int k) {
  if (k == 0) return 1.0;
  const int n = S.n;
  long long t = ((long long)k * (long long)L) % n;
  if (t > n - t) t = n - t;
  const double num = S.sin64[t];
  const double den = (double)L * S.sin64[k];
  double w = (num / den) * (num / den);
  return w > 1.0 ? 1.0 : (w < 0.0 ? 0.0 : w);
}

// w_hat_k, 1 - w_hat_k and log2(1 - w_hat_k) in binary64: the closed form for
// the triangle, the plan's binary64 row of 1 - w_hat_k for a shape window.
struct W64 {
  double w, om, hl;
};

__device__ __forceinline__ W64 win64(const FftSched& S, int L, int k) {
  if (S.om64) {
    const double om = S.om64[(size_t)(L - 1) * (size_t)S.om64_stride + k];
    return W64{1.0 - om, om, log2(om)};
  }
  const double w = what64(S, L, k);
  return W64{w, 1.0 - w, log1p(-w) * 1.4426950408889634};
}

// ---------------------------------------------- shape-generated windows
// The window generated by a shape g (Theorem 4's double convolution, eq.
// W_m): filter h_i = g((i + 1/2)/L), i < L, g the piecewise-linear interpolant
// of glen equispaced samples on [0, 1]; w_hat_k = |H_k|^2 / H_0^2.

// Bins with 1 - w_hat below this are taken from shape_om_direct.
constexpr double kShapeDirectBelow = 1.0 / 4096.0;

__device__ __forceinline__ double shape_tap(const double* __restrict__ g, int glen, int L, int i) {
  if (glen == 1) return g[0];
  const double t = ((double)i + 0.5) / (double)L * (double)(glen - 1);
  int j = (int)floor(t);
  if (j > glen - 2) j = glen - 2;
  const double f = t - (double)j;
  return (1.0 - f) * g[j] + f * g[j + 1];
}

__device__ __forceinline__ ff ff_from_double(double v) {
  const float hi = (float)v;
  return ff{hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// 1 - w_hat_k in binary64 without cancellation next to DC, for one bin k >= 1,
// by the 32 lanes of a warp together (every lane gets the result).  With the
// phase centred on the centroid c of h (inv = 1 / sum h):
//   H_0^2 - |H_k|^2 = (H_0 - C)(H_0 + C) - S^2,
//   H_0 - C = 2 sum_i h_i sin^2(pi k (i - c)/n),  S = sum_i h_i sin(2 pi k (i - c)/n),
// where S is third order in k (i - c)/n, so nothing cancels.
__device__ __forceinline__ double shape_om_direct(const double* __restrict__ g, int glen, int L,
                                                  int n, int k, double c, double inv) {
  const int lane = threadIdx.x & 31;
  const double kc = fmod((double)k * c, (double)n);  // common phase: its rounding cancels in |H_k|
  double A = 0.0, Sk = 0.0;
  for (int i = lane; i < L; i += 32) {
    const double h = shape_tap(g, glen, L, i) * inv;
    double u = ((double)(((long long)k * (long long)i) % n) - kc) / (double)n;
    u -= rint(u);  // k (i - c)/n reduced to [-1/2, 1/2]: sin^2 and sin(2 pi u) keep their values
    double sn, cs;
    sincospi(u, &sn, &cs);
    A += h * sn * sn;
    Sk += 2.0 * h * sn * cs;
  }
  A = warp_reduce(A, OpAdd());
  Sk = warp_reduce(Sk, OpAdd());
  // (H_0 - C)(H_0 + C) - S^2 with H_0 = 1, H_0 - C = 2A, H_0 + C = 2 - 2A
  const double om = 4.0 * A * (1.0 - A) - Sk * Sk;
  return om < 0.0 ? 0.0 : (om > 1.0 ? 1.0 : om);
}

// g = (1 - w_hat)^m = 2^(m log2(1 - w_hat)) and 1 - g; 1 - g from expm1 when
// g is close to 1, where 1 - g would cancel.
__device__ __forceinline__ void multiplier(int m, float hl, float& g, float& omg) {
  const float e = (float)m * hl;
  g = exp2f(e);
  omg = e > -1.f ? -expm1f(e * 0.693147180559945309f) : 1.f - g;
}

// Thresholded IMF (eq. I_gamma, eq. IMF_cont_stop_threshold): bin k passes
// whole (w_hat_k taken as 0) when (1 - w_hat_k)^m >= 1 - gamma.  Decided in
// FP32 on m log2(1 - w_hat_k) against log2(1 - gamma) outside the rounding
// band of both sides (table value good to 4u, the product u/2, the rounded
// log2(1 - gamma) u/2: band 8u (|x| + |c|)), else in binary64 (the sine
// table, or the shape window's binary64 row), as the binary64 definition
// decides.
__device__ __forceinline__ bool passes_whole(int m, float hl, const FftSched& S, int L, int k,
                                             const MethodParams& mp) {
  const float x = (float)m * hl, c = mp.log2_keep;
  if (x == -INFINITY) return false;  // w_hat = 1
  const float band = 8.f * 5.9604645e-8f * (fabsf(x) + fabsf(c)) + 1e-30f;
  if (x > c + band) return true;
  if (x < c - band) return false;
  return pow(win64(S, L, k).om, (double)m) >= 1.0 - mp.gamma;
}

__device__ __forceinline__ void multiplier_th(int m, float hl, const FftSched& S, int L, int k,
                                              const MethodParams& mp, float& g, float& omg) {
  multiplier(m, hl, g, omg);
  if (mp.threshold && passes_whole(m, hl, S, L, k, mp)) {
    g = 1.f;
    omg = 0.f;
  }
}

// --------------------------------------------------------- m selection

struct MSelState {
  float sc;      // power-of-two scale of the spectrum (|sc r_k| <= 1 for every k)
  int flags;
};

// Power of two sc with n * smax * sc <= 1: bounds every bin |r_k| <= n max|s|.
__device__ __forceinline__ float spectrum_scale(int n, float smax) {
  const float b = (float)n * smax;
  if (!(b > 0.f)) return 1.f;
  int e;
  frexpf(b, &e);  // b < 2^e
  return ldexpf(1.f, -e);
}

// SD_j in binary64 (Parseval, eq. SD), log-domain normalised so that no
// weight under- or overflows: weight_k = c_k |r_k|^2 (1 - w_k)^{2(j-1)}.
static __device__ double exact_sd(const float2* spec, const FftSched& S, int L, int j, RedScratch* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double M = -INFINITY, dummy = -INFINITY;
  for (int k = tid; k < S.P; k += nt) {
    const float2 z = spec[k];
    const double q = (double)parseval_weight(S, k) * ((double)z.x * z.x + (double)z.y * z.y);
    if (q > 0.0) {
      double lw = log2(q);
      if (j > 1) lw += 2.0 * (j - 1) * win64(S, L, k).hl;
      M = fmax(M, lw);
    }
  }
  block_reduce2(M, dummy, OpMax(), (double)-INFINITY, red);
  double num = 0.0, den = 0.0;
  if (M > -INFINITY) {
    for (int k = tid; k < S.P; k += nt) {
      const float2 z = spec[k];
      const double q = (double)parseval_weight(S, k) * ((double)z.x * z.x + (double)z.y * z.y);
      if (q > 0.0) {
        const W64 v = win64(S, L, k);
        double lw = log2(q);
        if (j > 1) lw += 2.0 * (j - 1) * v.hl;
        const double e = exp2(lw - M);
        den += e;
        num += e * v.w * v.w;
      }
    }
  }
  block_reduce2(num, den, OpAdd(), 0.0, red);
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

// One-pass sums of the FP32 screen of SD_j, all relative to 2^M: den =
// sum_k qw_k and num = sum_k qw_k w_k^2 with qw_k the weight of bin k, and the
// error weights aden = sum_k qw_k |e_k|, anum = sum_k qw_k w_k^2 |e_k|.
struct Online {
  float M, num, den, anum, aden;
};

// Binades a term may exceed the running reference exponent of the one-pass
// screen before the sums are rescaled.
constexpr float kLazyRescale = 32.f;

// Bins whose loads a thread issues together in the screen and the multiplier.
constexpr int kSdBatch = 4;

__device__ __forceinline__ Online online_merge(Online a, Online b) {
  if (a.M < b.M) {
    const Online t = a;
    a = b;
    b = t;
  }
  if (b.M == -INFINITY) return a;
  const float s = exp2f(b.M - a.M);
  return Online{a.M, fmaf(b.num, s, a.num), fmaf(b.den, s, a.den), fmaf(b.anum, s, a.anum),
                fmaf(b.aden, s, a.aden)};
}

// q = qm 2^qe exactly, qe an integer in [-127, 1] for 0 < q < 4: the
// exponent field of a normal q, and -127 with qm = q 2^127 (normal) for a
// subnormal one.
__device__ __forceinline__ void q_split(float q, float& qm, float& qe) {
  const int b = __float_as_int(q);
  const int ex = (b >> 23) & 0xff;
  if (ex != 0) {
    qm = __int_as_float((b & 0x007fffff) | 0x3f800000);
    qe = (float)(ex - 127);
  } else {
    qm = q * 1.7014118346046923e38f;  // 2^127
    qe = -127.f;
  }
}

// Term k of the screen for any scale of the spectrum: qw_k = qm_k 2^(t_k - M)
// with q_k = c_k |sc r_k|^2 = qm_k 2^(qe_k), t_k = e_k + qe_k, e_k =
// 2(j-1) log2(1-w_k), and M a running reference raised to t_k whenever t_k
// exceeds it by more than kLazyRescale (the sums are rescaled then).  Every
// term is below 2^(kLazyRescale+1), the largest is at least 2^-22, and no
// intermediate overflows; a term that underflows is below 2^-126 of the
// largest.
__device__ __forceinline__ void sd_term(float qm, float qe, float e, float w2, Online& o) {
  const float t = e + qe;
  if (t > o.M + kLazyRescale) {
    const float s = exp2f(o.M - t);  // 0 when o.M = -inf
    o.num *= s;
    o.den *= s;
    o.anum *= s;
    o.aden *= s;
    o.M = t;
  }
  const float qw = qm * exp2f(t - o.M);
  const float qwe = qw * fabsf(e);
  o.den += qw;
  o.num = fmaf(qw, w2, o.num);
  o.aden += qwe;
  o.anum = fmaf(qwe, w2, o.anum);
}

// Error band of the FP32 ratio num/den relative to the binary64 SD_j^2 on the
// same spectrum (u = 2^-24), for sums built from per-thread chains of at most
// `chain` terms combined over at most `levels` merge steps.
//
// The weight of term k is 2^(x_k) qm_k with x_k = (e_k + qe_k) - M computed in
// FP32 from hl_k = log2(1 - w_hat_k), a table value good to 4u relative
// (binary64 rounded, or the float-float row of the multi-pass path).  The
// error of x_k is at most (table) 4u|e_k| + (product 2(j-1) hl_k) u/2 |e_k|
// + (sum) u/2 (|e_k| + |qe_k|) + (difference) u/2 |x_k| <= 5u|e_k| + 139u
// (|qe_k| <= 127, |x_k| <= 150 on every term above 2^-150 of the largest),
// ln2 times that on the weight.  Weighted over the sums this is
// ln2 u (5 aden/den + 139) for den and ln2 u (5 anum/num + 139) for num,
// measured on the data (a posteriori).  exp2f adds 2 ulp and the product with
// qm u/2; each running rescale (at most one per term of a chain and one per
// merge step) 2 ulp; w^2, |r|^2 and the division 8u together; the summation
// of positive terms (chain + levels + 2) u per sum.  The band is four times
// the total.
__host__ __device__ __forceinline__ float screen_margin(const Online& r, float chain, float levels) {
  const float u = 5.9604645e-8f, c = 0.6931472f * u;
  const float ed = r.aden / r.den;
  const float en = r.num > 0.f ? r.anum / r.num : 0.f;
  const float resc = 2.5f * u + 4.f * u * (chain + levels);
  const float wden = c * (5.f * ed + 139.f) + resc;
  const float wnum = c * (5.f * en + 139.f) + resc;
  const float serr = (chain + levels + 2.f) * u;
  return 4.f * (wden + wnum + 2.f * serr + 8.f * u);
}

// Take the decision SD_j < delta from the FP32 sums if the ratio lies
// outside their error band, else re-take it on the binary64 value.
static __device__ bool decide_sd(const Online& r, float chain, float levels, const float2* spec,
                                 const FftSched& S, int L, int j, const MethodParams& mp,
                                 MSelState& st, RedScratch* red) {
  const float d2 = mp.delta2;
  const float ratio = r.num / r.den;
  if (r.den >= 0.5f && ratio == ratio) {
    const float margin = screen_margin(r, chain, levels);
    if (ratio <= d2 * (1.f - margin)) return true;
    if (ratio >= d2 * (1.f + margin)) return false;
  }
  const double sd = exact_sd(spec, S, L, j, red);
  st.flags |= FIF_FLAG_FP64_TIEBREAK;
  if (fabs(sd - mp.delta) <= 1e-6 * mp.delta) st.flags |= FIF_FLAG_NEAR_DELTA_TIE;
  return sd < mp.delta;
}

// Sums of one warp relative to a common reference: the warp's largest M (a
// max-reduction), each lane's sums rescaled once by 2^(M_lane - M), then
// plain sums.  Every lane gets the result.
__device__ __forceinline__ Online warp_merge(Online o) {
  float M = o.M;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, off));
  const float s = o.M == -INFINITY ? 0.f : exp2f(o.M - M);  // <= 1; an empty lane adds 0
  float num = o.num * s, den = o.den * s, anum = o.anum * s, aden = o.aden * s;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, off);
    den += __shfl_xor_sync(0xffffffffu, den, off);
    anum += __shfl_xor_sync(0xffffffffu, anum, off);
    aden += __shfl_xor_sync(0xffffffffu, aden, off);
  }
  return Online{M, num, den, anum, aden};
}

// Block-wide merge of the per-thread sums (two levels of warp_merge: at most
// one rescale and five summation levels each); every thread gets the result.
__device__ __forceinline__ Online online_block_reduce(Online o, RedScratch* red) {
  o = warp_merge(o);
  float* s = reinterpret_cast<float*>(red->d);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    s[5 * wid] = o.M;
    s[5 * wid + 1] = o.num;
    s[5 * wid + 2] = o.den;
    s[5 * wid + 3] = o.anum;
    s[5 * wid + 4] = o.aden;
  }
  __syncthreads();
  Online r = lane < nw ? Online{s[5 * lane], s[5 * lane + 1], s[5 * lane + 2], s[5 * lane + 3],
                                s[5 * lane + 4]}
                       : Online{-INFINITY, 0.f, 0.f, 0.f, 0.f};
  return warp_merge(r);
}

// FP32 screen of SD_j < delta over the bins in one CTA pass (sd_term per
// bin), then the decision.
static __device__ bool sd_below(const float2* spec, const FftSched& S, const float2* row, int L,
                                int j, const MethodParams& mp, MSelState& st, RedScratch* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const float e2 = 2.f * (float)(j - 1);
  Online o{-INFINITY, 0.f, 0.f, 0.f, 0.f};
  // kSdBatch bins per step, their loads issued together (the row lives in
  // global memory or L2 for most callers)
  for (int k0 = tid; k0 < S.P; k0 += kSdBatch * nt) {
    float2 z[kSdBatch], tv[kSdBatch];
#pragma unroll
    for (int u = 0; u < kSdBatch; u++) {
      const int k = k0 + u * nt;
      z[u] = k < S.P ? spec[k] : make_float2(0.f, 0.f);
      tv[u] = k < S.P ? row[k] : make_float2(0.f, 0.f);  // global (plan table, multi-pass row)
    }
#pragma unroll
    for (int u = 0; u < kSdBatch; u++) {
      const int k = k0 + u * nt;
      const float re = z[u].x * st.sc, im = z[u].y * st.sc;
      const float q = parseval_weight(S, k) * fmaf(re, re, im * im);
      if (!(q > 0.f)) continue;  // also zero bins and bins past the end
      const float e = (j == 1) ? 0.f : e2 * tv[u].x;
      if (e == -INFINITY) continue;  // w_hat = 1 (the DC bin): weight 0 for j > 1
      float qm, qe;
      q_split(q, qm, qe);
      sd_term(qm, qe, e, tv[u].y * tv[u].y, o);
    }
  }
  const Online r = online_block_reduce(o, red);
  // chain: bins per thread; levels: the warp and CTA trees
  const float chain = (float)((S.P + nt - 1) / nt);
  return decide_sd(r, chain, 10.f, spec, S, L, j, mp, st, red);
}

// A-priori mode (Theorem 5, eq. N0_discrete): m = the least natural N0 with
// N0^N0 / (N0+1)^(N0+1) < delta / (||U^T r||_inf sqrt(n - 1 - k)), capped at
// max_inner.  ||U^T r||_inf = max_k |r_hat_k| / sqrt(n) over the half spectrum
// (a real signal's other bins mirror it); k = gcd(n, L) - 1 is the number of
// zero eigenvalues of W (w_hat_k = 0 exactly where kL = 0 mod n, k != 0).
// The bound is decided on one thread, in logs (log f(N) = N log N -
// (N+1) log(N+1), decreasing in N), every comparison with the binary64
// answer (N0Test); a left side within 1e-6 of the right at a tested N is
// flagged NEAR_DELTA_TIE.
__device__ __forceinline__ double n0_lhs(int N) {
  return (double)N * log((double)N) - (double)(N + 1) * log((double)(N + 1));
}

// The comparison lhs(N) < rhs of the bound: in FP32 (stable form
// -log1p(N) - N log1p(1/N), absolute error below 1e-5 on both sides) when the
// two sides are more than 1e-4 apart, else re-taken in binary64 (where a
// difference within 1e-6 raises the tie flag).  Same answer as binary64.
struct N0Test {
  float rhs_f;
  double rhs_d;
  int flags;
  __device__ bool below(int N) {
    const float x = (float)N;
    const float lf = -log1pf(x) - x * log1pf(1.f / x);
    if (fabsf(lf - rhs_f) > 1e-4f) return lf < rhs_f;
    const double ld = n0_lhs(N);
    if (fabs(ld - rhs_d) <= 1e-6) flags |= FIF_FLAG_NEAR_DELTA_TIE;
    return ld < rhs_d;
  }
};

static __device__ int apriori_m(const float2* spec, const FftSched& S, int L, const MethodParams& mp,
                                int& flags, RedScratch* red) {
  float mx = 0.f;
  for (int k = threadIdx.x; k < S.P; k += blockDim.x) {
    const float2 z = spec[k];
    mx = fmaxf(mx, fmaf(z.x, z.x, z.y * z.y));
  }
  float dummy = 0.f;
  block_reduce2(mx, dummy, OpMax(), 0.f, red);
  __syncthreads();  // every thread has read red before thread 0 reuses it
  int* out = reinterpret_cast<int*>(red->d);
  if (threadIdx.x == 0) {
    int a = S.n, b = L;
    while (b) {
      const int t = a % b;
      a = b;
      b = t;
    }
    const long long dof = (long long)S.n - 1 - (a - 1);
    const int jmax = mp.max_inner;
    int N0 = 1;
    N0Test t{0.f, 0.0, 0};
    if (mx > 0.f && dof > 0) {
      // rhs = log delta - log ||U^T r||_inf - log sqrt(dof), ||U^T r||_inf = sqrt(mx / n)
      t.rhs_d = log(mp.delta) - 0.5 * (log((double)mx) - log((double)S.n)) - 0.5 * log((double)dof);
      t.rhs_f = (float)t.rhs_d;
      if (!t.below(jmax)) {
        N0 = jmax + 1;
      } else {
        // log f(N) = -log(N+1) - 1 + O(1/N): start from N + 1 = exp(-rhs - 1),
        // step to the least N that passes, bisect if the estimate is far off
        const float est = expf(-t.rhs_f - 1.f) - 1.f;
        int g = est >= (float)jmax ? jmax : (est <= 1.f ? 1 : (int)est);
        int steps = 0;
        while (g > 1 && t.below(g - 1) && steps < 8) g--, steps++;
        while (!t.below(g) && steps < 16) g++, steps++;
        if (!(t.below(g) && (g == 1 || !t.below(g - 1)))) {
          int lo = 0, hi = jmax;  // lhs(lo) >= rhs (lhs(0) = 0 >= rhs here), lhs(hi) < rhs
          if (t.below(1)) hi = 1;
          while (hi - lo > 1) {
            const int mid = lo + (hi - lo) / 2;
            if (t.below(mid))
              hi = mid;
            else
              lo = mid;
          }
          g = hi;
        }
        N0 = g;
      }
    }
    int f = t.flags;
    if (N0 > jmax) {
      N0 = jmax;
      f |= FIF_FLAG_MAX_INNER_HIT;
    }
    out[0] = N0;
    out[1] = f;
  }
  __syncthreads();
  const int m = out[0];
  flags |= out[1];
  __syncthreads();  // before red is reused
  return m;
}

// m = first j in [1, max_inner] with SD_j < delta, else max_inner (eq. SD,
// Sec. 4).  SD_j is non-increasing in j (raising j reweights towards bins
// with small w_hat, where w_hat^2 is small), so the first crossing is found by
// testing j = max_inner, then bisecting.
static __device__ int select_m(const float2* spec, const FftSched& S, int L, const MethodParams& mp,
                               float sc, int& flags, RedScratch* red) {
  if (mp.apriori) return apriori_m(spec, S, L, mp, flags, red);
  const float2* row = wrow(S, L);
  MSelState st;
  st.sc = sc;
  st.flags = 0;
  int m;
  const int jmax = mp.max_inner;
  if (!sd_below(spec, S, row, L, jmax, mp, st, red)) {
    m = jmax;
    st.flags |= FIF_FLAG_MAX_INNER_HIT;
  } else {
    int lo = 0, hi = jmax;
    while (hi - lo > 1) {
      const int mid = lo + (hi - lo) / 2;
      if (sd_below(spec, S, row, L, mid, mp, st, red))
        hi = mid;
      else
        lo = mid;
    }
    m = hi;
  }
  flags |= st.flags;
  return m;
}

// The multiplier pairs {(1 - w_hat_k)^m, 1 - (1 - w_hat_k)^m} of every bin for
// this m (thresholded when gamma > 0) into mult[0..P).
static __device__ void multiplier_pass(float2* mult, const FftSched& S, const float2* row, int L,
                                       int m, const MethodParams& mp) {
  const int nt = blockDim.x;
  for (int k0 = threadIdx.x; k0 < S.P; k0 += kSdBatch * nt) {
    float hl[kSdBatch];
#pragma unroll
    for (int u = 0; u < kSdBatch; u++) {
      const int k = k0 + u * nt;
      hl[u] = k < S.P ? __ldg(&row[k].x) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kSdBatch; u++) {
      const int k = k0 + u * nt;
      if (k >= S.P) break;
      float g, omg;
      multiplier_th(m, hl[u], S, L, k, mp, g, omg);
      mult[k] = make_float2(g, omg);
    }
  }
  __syncthreads();
}

// m of eq. SD (or the a-priori bound) as select_m, and where the IMF's
// multiplier pairs are for inverse_real_mult (src): for m = max_inner, the
// usual outcome, the plan's table row (S.gtab, binary64-rounded), else a
// pass that writes them into mult[0..P).  (Computing the
// pairs inside the first screen pass, speculatively for m = max_inner, was
// measured slower: the longer loop body spills at 64 registers a thread.)
static __device__ int select_m_mult(const float2* spec, float2* mult, const FftSched& S, int L,
                                    const MethodParams& mp, float sc, int& flags,
                                    RedScratch* red, const float2*& src) {
  const float2* row = wrow(S, L);
  const float2* grow = S.gtab ? S.gtab + (size_t)(L - 1) * (size_t)S.P : nullptr;
  src = mult;
  if (mp.apriori) {
    const int m = apriori_m(spec, S, L, mp, flags, red);
    if (grow && m == mp.max_inner)
      src = grow;
    else
      multiplier_pass(mult, S, row, L, m, mp);
    return m;
  }
  MSelState st;
  st.sc = sc;
  st.flags = 0;
  int m;
  const int jmax = mp.max_inner;
  if (!sd_below(spec, S, row, L, jmax, mp, st, red)) {
    m = jmax;
    st.flags |= FIF_FLAG_MAX_INNER_HIT;
  } else {
    int lo = 0, hi = jmax;
    while (hi - lo > 1) {
      const int mid = lo + (hi - lo) / 2;
      if (sd_below(spec, S, row, L, mid, mp, st, red))
        hi = mid;
      else
        lo = mid;
    }
    m = hi;
  }
  if (grow && m == jmax)
    src = grow;  // the plan's table row: no pass
  else
    multiplier_pass(mult, S, row, L, m, mp);
  flags |= st.flags;
  return m;
}

// select_m on an explicit window row (row[k] = {log2(1 - w_hat_k), w_hat_k} for
// the current L), for paths that compute the row per IMF instead of keeping
// the whole table.
static __device__ int select_m_on_row(const float2* spec, const FftSched& S, const float2* row,
                                      int L, const MethodParams& mp, float sc, int& flags,
                                      RedScratch* red) {
  if (mp.apriori) return apriori_m(spec, S, L, mp, flags, red);
  MSelState st;
  st.sc = sc;
  st.flags = 0;
  int m;
  const int jmax = mp.max_inner;
  if (!sd_below(spec, S, row, L, jmax, mp, st, red)) {
    m = jmax;
    st.flags |= FIF_FLAG_MAX_INNER_HIT;
  } else {
    int lo = 0, hi = jmax;
    while (hi - lo > 1) {
      const int mid = lo + (hi - lo) / 2;
      if (sd_below(spec, S, row, L, mid, mp, st, red))
        hi = mid;
      else
        lo = mid;
    }
    m = hi;
  }
  flags |= st.flags;
  return m;
}

// Time-domain epilogue of one IMF: scale the inverse transform by 1/n, store
// the IMF row, subtract it from the remainder.  Returns ||IMF||_inf.
static __device__ float store_imf_update_rem(const float2* work, float* rem, float* out_row,
                                      const FftSched& S, RedScratch* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const float inv_n = 1.f / (float)S.n;
  float imax = 0.f;
  if (!S.odd) {
    for (int t = tid; t < S.Nc; t += nt) {
      const float2 z = work[t];
      const float a = z.x * inv_n, b = z.y * inv_n;
      out_row[2 * t] = a;
      out_row[2 * t + 1] = b;
      rem[2 * t] -= a;
      rem[2 * t + 1] -= b;
      imax = fmaxf(imax, fmaxf(fabsf(a), fabsf(b)));
    }
  } else {
    for (int t = tid; t < S.n; t += nt) {
      const float a = work[t].x * inv_n;
      out_row[t] = a;
      rem[t] -= a;
      imax = fmaxf(imax, fabsf(a));
    }
  }
  float dummy = 0.f;
  block_reduce2(imax, dummy, OpMax(), 0.f, red);
  return imax;
}

struct EpiOut {
  float imax;   // ||IMF||_inf
  int k;        // extrema of the new remainder
  int zc;       // zero crossings of the new remainder
  int tie;      // extrema tie (see count_extrema)
  float rmax;   // ||r||_inf of the new remainder
};

// Whether the extrema count could change when r moves by tau/2 around the
// difference d0 (neighbours dm, dp): d0 within tau of zero and either exactly
// zero (a plateau between a rise and a fall holds no extremum, and either
// sign of d0 makes one: a change of one), or a neighbour also within tau, or
// both neighbours of one sign (a flip of d0 adds or removes two).
__device__ __forceinline__ bool diff_tie(float dm, float d0, float dp, float tau) {
  return fabsf(d0) <= tau &&
         (d0 == 0.f || fabsf(dm) <= tau || fabsf(dp) <= tau || ((dm > 0.f) == (dp > 0.f)));
}

// Extrema, zero-crossing and tie terms owned by the sample pair (2t, 2t+1),
// given r[2t-1 .. 2t+3]: samples 2t and 2t+1, differences d_2t and d_2t+1,
// crossings (2t, 2t+1) and (2t+1, 2t+2).  Same definitions as count_extrema.
__device__ __forceinline__ void pair_terms(float rm1, float r0, float r1, float r2, float r3,
                                           float tau, int& ext, int& zc, int& tie) {
  const float dm1 = r0 - rm1, d0 = r1 - r0, d1 = r2 - r1, d2 = r3 - r2;
  ext += (dm1 > 0.f && d0 < 0.f) || (dm1 < 0.f && d0 > 0.f);
  ext += (d0 > 0.f && d1 < 0.f) || (d0 < 0.f && d1 > 0.f);
  zc += (r0 > 0.f && r1 < 0.f) || (r0 < 0.f && r1 > 0.f);
  zc += (r1 > 0.f && r2 < 0.f) || (r1 < 0.f && r2 > 0.f);
  tie |= diff_tie(dm1, d0, d1, tau);
  tie |= diff_tie(d0, d1, d2, tau);
}

// Time-domain epilogue of one IMF (even n) fused with the extrema count of
// the new remainder.  Pass 1: the thread of point t (samples 2t, 2t+1) scales
// the inverse transform by 1/n, stores the IMF row, writes r <- r - IMF, and
// takes the terms of its pair from its neighbours' new values by warp
// shuffles.  Pass 2 (after a barrier): the pairs at the edges of each block
// of 32 points (and the last pair) take their terms from memory.
static __device__ EpiOut epilogue_extrema_even(const float2* work, float* rem, float* out_row,
                                               const FftSched& S, float tau, RedScratch* red) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const int Nc = S.Nc, n = S.n;
  const float inv_n = 1.f / (float)n;
  const bool vec = (reinterpret_cast<uintptr_t>(out_row) & 7) == 0;
  float imax = 0.f, rmax = 0.f;
  int ext = 0, zc = 0, tie = 0;
  for (int base = tid - lane; base < Nc; base += nt) {
    const int t = base + lane;
    const bool act = t < Nc;
    float ra = 0.f, rb = 0.f;
    if (act) {
      const float2 z = work[t];
      const float a = z.x * inv_n, b = z.y * inv_n;
      if (vec) {
        *reinterpret_cast<float2*>(out_row + 2 * t) = make_float2(a, b);
      } else {
        out_row[2 * t] = a;
        out_row[2 * t + 1] = b;
      }
      // one 8-byte access per lane: conflict-free, where two scalar ones are 2-way
      const float2 rr = *reinterpret_cast<const float2*>(rem + 2 * t);
      ra = rr.x - a;
      rb = rr.y - b;
      *reinterpret_cast<float2*>(rem + 2 * t) = make_float2(ra, rb);
      imax = fmaxf(imax, fmaxf(fabsf(a), fabsf(b)));
      rmax = fmaxf(rmax, fmaxf(fabsf(ra), fabsf(rb)));
    }
    const float p_rb = __shfl_up_sync(0xffffffffu, rb, 1);
    const float n_ra = __shfl_down_sync(0xffffffffu, ra, 1);
    // the pair's extrema and crossings (as pair_terms); its tie test only in the
    // rare warps where one of its two differences lies within tau of zero
    const bool in = act && lane != 0 && lane != 31 && t != Nc - 1;
    const float dm1 = ra - p_rb, d0 = rb - ra, d1 = n_ra - rb;
    if (in) {
      ext += (dm1 > 0.f && d0 < 0.f) || (dm1 < 0.f && d0 > 0.f);
      ext += (d0 > 0.f && d1 < 0.f) || (d0 < 0.f && d1 > 0.f);
      zc += (ra > 0.f && rb < 0.f) || (ra < 0.f && rb > 0.f);
      zc += (rb > 0.f && n_ra < 0.f) || (rb < 0.f && n_ra > 0.f);
    }
    if (__any_sync(0xffffffffu, in && (fabsf(d0) <= tau || fabsf(d1) <= tau))) {
      const float n_rb = __shfl_down_sync(0xffffffffu, rb, 1);
      if (in) tie |= diff_tie(dm1, d0, d1, tau) || diff_tie(d0, d1, n_rb - n_ra, tau);
    }
  }
  __syncthreads();
  const int nblk = (Nc + 31) >> 5;
  for (int i = tid; i < 2 * nblk; i += nt) {
    const int b0 = (i >> 1) << 5;
    const int t = (i & 1) ? min(b0 + 31, Nc - 1) : b0;
    if ((i & 1) && t == b0) continue;
    const int s0 = 2 * t;
    const float rm1 = rem[s0 == 0 ? n - 1 : s0 - 1];
    const float r0 = rem[s0], r1 = rem[s0 + 1];
    const float r2 = rem[s0 + 2 >= n ? s0 + 2 - n : s0 + 2];
    const float r3 = rem[s0 + 3 >= n ? s0 + 3 - n : s0 + 3];
    pair_terms(rm1, r0, r1, r2, r3, tau, ext, zc, tie);
  }
  // one block-wide merge of the five results (two barriers)
  float fe = (float)ext, fz = (float)zc;  // exact: counts < 2^24
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fe += __shfl_xor_sync(0xffffffffu, fe, off);
    fz += __shfl_xor_sync(0xffffffffu, fz, off);
    imax = fmaxf(imax, __shfl_xor_sync(0xffffffffu, imax, off));
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
  }
  tie = __any_sync(0xffffffffu, tie);
  float* sm = reinterpret_cast<float*>(red->d);
  const int wid = tid >> 5, nw = (nt + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    sm[5 * wid] = fe;
    sm[5 * wid + 1] = fz;
    sm[5 * wid + 2] = imax;
    sm[5 * wid + 3] = rmax;
    sm[5 * wid + 4] = tie ? 1.f : 0.f;
  }
  __syncthreads();
  fe = lane < nw ? sm[5 * lane] : 0.f;
  fz = lane < nw ? sm[5 * lane + 1] : 0.f;
  imax = lane < nw ? sm[5 * lane + 2] : 0.f;
  rmax = lane < nw ? sm[5 * lane + 3] : 0.f;
  float ft = lane < nw ? sm[5 * lane + 4] : 0.f;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fe += __shfl_xor_sync(0xffffffffu, fe, off);
    fz += __shfl_xor_sync(0xffffffffu, fz, off);
    imax = fmaxf(imax, __shfl_xor_sync(0xffffffffu, imax, off));
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
    ft = fmaxf(ft, __shfl_xor_sync(0xffffffffu, ft, off));
  }
  EpiOut o;
  o.imax = imax;
  o.k = (int)fe;
  o.zc = (int)fz;
  o.tie = ft > 0.f;
  o.rmax = rmax;
  return o;
}

struct ExtremaInfo {
  int k;
  int zc;
  int tie;
  float rmax;
};

// Periodic extrema count (index i with d_{i-1} d_i < 0, d_i = r_{i+1} - r_i),
// zero crossings, and whether the count could change under a perturbation of
// r of tau/2 (some |d_i| <= tau whose flip would add or remove a pair).
static __device__ ExtremaInfo count_extrema(const float* rem, int n, float tau, RedScratch* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int ext = 0, zc = 0, tie = 0;
  float rmax = 0.f;
  for (int i = tid; i < n; i += nt) {
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
  float fe = (float)ext, fz = (float)zc;  // exact: counts < 2^24
  block_reduce2(fe, fz, OpAdd(), 0.f, red);
  float dummy = 0.f;
  block_reduce2(rmax, dummy, OpMax(), 0.f, red);
  ExtremaInfo e;
  e.k = (int)fe;
  e.zc = (int)fz;
  e.tie = tie;
  e.rmax = rmax;
  return e;
}

// Outer-loop test before IMF K (Algorithm 2 "while #extrema >= 2", the
// max_imfs cap, the window limit 2L-1 <= n).  Returns 0 and sets L to
// continue, else the stop reason.  Same value in every thread.
// Fourier-peak mask length (end of Sec. 2): k* = the largest |r_hat_k| over
// 1 <= k <= n/2 (smallest k among equal magnitudes) and whether another bin
// lies within 1e-5 (relative, on |r_hat|^2) of it.  One CTA over the half
// spectrum; every thread gets the result.  The key packs the FP32 magnitude
// (non-negative: its bits order as integers) above the complemented index.
struct SpecPeak {
  int k;
  int tie;
};

__device__ __forceinline__ unsigned long long peak_key(float v, int k) {
  return ((unsigned long long)__float_as_uint(v) << 32) | (unsigned)(0xffffffffu - (unsigned)k);
}

static __device__ SpecPeak spectral_peak(const float2* spec, const FftSched& S, RedScratch* red) {
  unsigned long long best = 0ull;
  for (int k = 1 + threadIdx.x; k < S.P; k += blockDim.x) {
    const float2 z = spec[k];
    const unsigned long long key = peak_key(fmaf(z.x, z.x, z.y * z.y), k);
    best = key > best ? key : best;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  unsigned long long* sm = reinterpret_cast<unsigned long long*>(red->d);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sm[wid] = best;
  __syncthreads();
  best = lane < nw ? sm[lane] : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  SpecPeak r;
  r.k = best ? (int)(0xffffffffu - (unsigned)(best & 0xffffffffull)) : 0;
  const float vmax = __uint_as_float((unsigned)(best >> 32));
  int tie = 0;
  for (int k = 1 + threadIdx.x; k < S.P; k += blockDim.x) {
    const float2 z = spec[k];
    tie |= k != r.k && fmaf(z.x, z.x, z.y * z.y) >= vmax * (1.f - 1e-5f) && vmax > 0.f;
  }
  r.tie = __syncthreads_or(tie);
  return r;
}

// Under FIF_PEAK_MASK, L comes from the spectral peak k* (peak >= 1): the same
// rule at the count of extrema a tone of k* cycles has, 2 k*; the extrema
// count k still decides the stop.
__device__ __forceinline__ int outer_test(int k, int K, int n, const MethodParams& mp,
                                          const int32_t* forced_L, int& L, int& flags,
                                          int peak = 0, const int* ltab = nullptr) {
  if (mp.force_L) {
    if (K == mp.max_imfs) return FIF_STOP_MAX_IMFS;
    L = forced_L[K];
    if (L <= 0) return FIF_STOP_FORCED_END;
    if (2LL * L - 1 > n) return FIF_STOP_MASK;
    return 0;
  }
  if (k < 2) return FIF_STOP_EXTREMA;
  const int kk = mp.peak_mask ? 2 * (peak > 0 ? peak : 1) : k;
  if (ltab) {
    L = ltab[kk];  // the same binary64 rule, tabulated per length on the host
  } else {
    double t = mp.nu * (double)n;
    t = t / (double)kk;
    L = mp.mask_scale * (int)floor(t);
  }
  if (L < 2) {
    L = 2;
    flags |= FIF_FLAG_L_CLAMPED;
  }
  if (2LL * L - 1 > n) return FIF_STOP_MASK;
  if (K == mp.max_imfs) return FIF_STOP_MAX_IMFS;
  return 0;
}

// Perturbation threshold of the extrema tie test: 2^-17 max|s|.
__device__ __forceinline__ float tie_tau(float smax) { return smax * 7.62939453125e-06f; }

}  // namespace fif
