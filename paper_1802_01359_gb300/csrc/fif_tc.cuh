// Split-BF16 tensor-core radix-16 DFT stage (the FIF_PREC_SPLIT_BF16
// variant of the fused path's inverse FFT).
//
// A radix-16 Stockham pass multiplies, for every butterfly, the 16 twiddled
// inputs by the 16 x 16 DFT matrix F (F[r'][r] = exp(+-2 pi i r r'/16)).  In
// real form, with the inputs' real parts in rows 0..15 and imaginary parts in
// rows 16..31 of a 32 x 8 block (eight butterflies as columns):
//     [Re Y]   [Fr  -Fi] [Re X]
//     [Im Y] = [Fi   Fr] [Im X],
// four 16 x 16 x 8 products per eight butterflies, each one warp-level
// mma.m16n8k16 with BF16 operands and FP32 accumulation.  BF16 keeps 8
// significant bits, so both F and X are split into hi + lo (hi = bf16(x),
// lo = bf16(x - hi), together good to about 2^-18 relative) and each product
// is accumulated as hi*hi + hi*lo + lo*hi (the lo*lo term, about 2^-18 of the
// product, is dropped).  The result is within a few times 2^-18 of the FP32
// butterfly's, against 2^-24 for FP32 arithmetic; the measured IMF error is
// reported beside the FP32 path's.
//
// Fragment layout of mma.m16n8k16 (g = lane / 4, t = lane % 4): A (16 x 16,
// row major) register i holds rows g + 8 (i & 1), columns 2t + 8 (i >> 1) and
// the next one; B (16 x 8) register i holds rows 2t + 8 i and 2t + 8 i + 1 of
// column g; C/D holds rows g and g + 8, columns 2t and 2t + 1.  The lower half
// of a packed register is the element with the smaller index.
#pragma once

#include <stdint.h>

#include "fif_device.cuh"

namespace fif {

// {bf16(b), bf16(a)} packed: a in the upper half, b in the lower (round to nearest).
__device__ __forceinline__ uint32_t bf16x2_pack(float lower, float upper) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(upper), "f"(lower));
  return d;
}
__device__ __forceinline__ float bf16_lower(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_upper(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// hi + lo split of a pair (lower, upper): hi = bf16 of each, lo = bf16 of the rest.
__device__ __forceinline__ void bf16x2_split(float lower, float upper, uint32_t& hi, uint32_t& lo) {
  hi = bf16x2_pack(lower, upper);
  lo = bf16x2_pack(lower - bf16_lower(hi), upper - bf16_upper(hi));
}

// d += a * b, m16n8k16, BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// cos(2 pi m / 16) for any integer m (m mod 16), from the constants the FP32
// butterflies use: |cos| over an octant period is 1, cos(pi/8), sqrt(1/2),
// sin(pi/8), 0.
__device__ __forceinline__ float cos16(int m) {
  m &= 15;
  const int a = m & 7;        // angle mod 180 degrees, in 22.5-degree steps
  const int b = a > 4 ? 8 - a : a;  // reflected into 0..4 (|cos| symmetric about 90)
  const float v = b == 0 ? 1.f : b == 1 ? Kc<float2>::c16() : b == 2 ? Kc<float2>::r2()
                : b == 3 ? Kc<float2>::s16() : 0.f;
  // cos < 0 for 90 < angle < 270 degrees: m in 5..11
  return (m > 4 && m < 12) ? -v : v;
}

// The lane's A fragments of Fr, Fi and -Fi (hi and lo) for the DFT direction.
struct TcDft16 {
  uint32_t fr_hi[4], fr_lo[4], fi_hi[4], fi_lo[4], nfi_hi[4], nfi_lo[4];
};

template <bool INV>
__device__ __forceinline__ TcDft16 tc_dft16_fragments() {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  TcDft16 A;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int row = g + 8 * (i & 1), col = 2 * t + 8 * (i >> 1);
    // F[r'][r] = exp(s 2 pi i r' r / 16), s = +1 inverse, -1 forward
    const int m0 = row * col, m1 = row * (col + 1);
    const float c0 = cos16(m0), c1 = cos16(m1);
    const float s0 = (INV ? 1.f : -1.f) * cos16(m0 - 4), s1 = (INV ? 1.f : -1.f) * cos16(m1 - 4);
    bf16x2_split(c0, c1, A.fr_hi[i], A.fr_lo[i]);
    bf16x2_split(s0, s1, A.fi_hi[i], A.fi_lo[i]);
    A.nfi_hi[i] = A.fi_hi[i] ^ 0x80008000u;  // exact: only the sign bits change
    A.nfi_lo[i] = A.fi_lo[i] ^ 0x80008000u;
  }
  return A;
}

// D += (Ahi + Alo)(Bhi + Blo) without the lo*lo term.
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ahi)[4], const uint32_t (&alo)[4],
                                     uint32_t bhi0, uint32_t bhi1, uint32_t blo0, uint32_t blo1) {
  mma_bf16_16816(d, ahi, bhi0, bhi1);
  mma_bf16_16816(d, ahi, blo0, blo1);
  mma_bf16_16816(d, alo, bhi0, bhi1);
}

// One radix-16 Stockham pass (E = 16: one butterfly per thread, T = Nc/16
// butterflies) on the tensor cores, in place.  Same data movement and
// twiddles as fft_pass<float2, INV, 16, 16>; the 16-point DFTs of each group
// of eight butterflies of a warp are the mma products above.  Every thread
// of the CTA calls it (the mma is warp-collective: lanes past T feed zeros
// and store nothing).
// lt: the thread's index among the S.T threads of this transform (several
// transforms may share a CTA; each must start on a warp boundary, T a
// multiple of 32 when there is more than one), S.T or more for threads
// without a butterfly.  The warp's first butterfly is lane 0's index (the
// same in every lane; T or more for a warp without butterflies).
// SWZ: the buffer is in the swizzled layout of S.swz (work_slot).
template <bool INV, bool SWZ = false>
__device__ __forceinline__ void fft_pass16_tc(float2* buf, const FftSched& S, const TwSrc& ts,
                                              int Ns, const TcDft16& A, int lt) {
  auto slot = [&](int i) { return SWZ ? work_slot(i, S.swz) : i; };
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int T = S.T, stride = S.Nc / 16, warp0 = __shfl_sync(0xffffffffu, lt, 0);
  const bool p2 = (Ns & (Ns - 1)) == 0;  // j mod Ns by a mask (2^a lengths)
  auto modNs = [&](int j) { return p2 ? (j & (Ns - 1)) : j % Ns; };
  // per group q: the butterfly of column g, inputs r = 2t, 2t+1, 2t+8, 2t+9
  float2 x[4][4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int jb = warp0 + 8 * q + g;
#pragma unroll
    for (int s = 0; s < 4; s++) {
      const int r = 2 * t + (s & 1) + 8 * (s >> 1);
      x[q][s] = jb < T ? buf[slot(jb + r * stride)] : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int jb = warp0 + 8 * q + g;
    const int k = modNs(jb);
    if (jb < T && k != 0) {
#pragma unroll
      for (int s = 0; s < 4; s++) {
        const int r = 2 * t + (s & 1) + 8 * (s >> 1);
        if (r == 0) continue;  // w^0 = 1
        float2 w;
        if (ts.p) {
          w = __ldg(ts.p + (Ns - 1) + (r - 1) * Ns + k);  // the per-pass table: inverse
          if (!INV) w = cconj(w);
        } else {
          w = tw_dir<INV>(ts, r * k * (S.n / (Ns * 16)));
        }
        x[q][s] = cmul(x[q][s], w);
      }
    }
    uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
    bf16x2_split(x[q][0].x, x[q][1].x, rh0, rl0);  // Re X, rows 2t, 2t+1
    bf16x2_split(x[q][2].x, x[q][3].x, rh1, rl1);  // Re X, rows 2t+8, 2t+9
    bf16x2_split(x[q][0].y, x[q][1].y, ih0, il0);  // Im X
    bf16x2_split(x[q][2].y, x[q][3].y, ih1, il1);
    float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
    mma3(yr, A.fr_hi, A.fr_lo, rh0, rh1, rl0, rl1);    // Re Y = Fr Re X
    mma3(yr, A.nfi_hi, A.nfi_lo, ih0, ih1, il0, il1);  //      - Fi Im X
    mma3(yi, A.fi_hi, A.fi_lo, rh0, rh1, rl0, rl1);    // Im Y = Fi Re X
    mma3(yi, A.fr_hi, A.fr_lo, ih0, ih1, il0, il1);    //      + Fr Im X
    // outputs r' = g (d[0], d[1]) and g + 8 (d[2], d[3]) of butterflies 2t, 2t+1
#pragma unroll
    for (int c = 0; c < 2; c++) {
      const int jo = warp0 + 8 * q + 2 * t + c;
      if (jo < T) {
        const int ko = modNs(jo);
        const int base = (jo - ko) * 16 + ko;
        buf[slot(base + g * Ns)] = make_float2(yr[c], yi[c]);
        buf[slot(base + (g + 8) * Ns)] = make_float2(yr[2 + c], yi[2 + c]);
      }
    }
  }
  __syncthreads();
}

// Complex FFT of S.Nc points with every radix-16 pass on the tensor cores
// (E = 16 schedules; the other passes as fft_inplace).
template <bool INV, bool SWZ = false>
__device__ __forceinline__ void fft_inplace_tc(float2* buf, const FftSched& S, const TwSrc& ts,
                                               int lt = threadIdx.x) {
  const TcDft16 A = tc_dft16_fragments<INV>();
  int Ns = 1;
#pragma unroll 1
  for (int p = 0; p < S.npass; p++) {
    const int R = S.radix[p];
    if (R == 16) {
      fft_pass16_tc<INV, SWZ>(buf, S, ts, Ns, A, lt);
    } else if (R == 8) {
      fft_pass<float2, INV, 8, 16, SWZ>(buf, S, ts, Ns, lt);
    } else {
      fft_tail_pass<float2, INV, 16, SWZ>(buf, S, ts, Ns, R, lt);
    }
    Ns *= R;
  }
}

// inverse_real_mult with the tensor-core FFT (E = 16).
__device__ __forceinline__ void inverse_real_mult_tc(float2* spec, float2* work, const float2* mult,
                                                     const FftSched& S, const TwSrc& ts) {
  inverse_real_mult_split(spec, work, mult, S, ts);
  fft_inplace_tc<true>(work, S, ts);
}

}  // namespace fif
