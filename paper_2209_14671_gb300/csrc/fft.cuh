// Device building blocks: complex arithmetic and a shared-memory Stockham FFT.
//
// A length-L transform is owned by a "team" of TL = min(32, L/8) lanes of one
// warp, so all of its synchronisation is __syncwarp().  Each pass reads the whole
// vector into registers (radix-R butterflies, R = 8 while possible, then 4 or 2),
// synchronises, and writes it back in Stockham (self-sorting) order, so the
// output is in natural order with no bit reversal.  Transforms are unnormalised:
// forward X[k] = sum_x x[x] e^{-2 pi i k x / L}, inverse with e^{+2 pi i k x / L}.
// Twiddles W_L^k = e^{-2 pi i k / L} come from a table built in FP64 on the host.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace elf {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* v);

template <>
__device__ __forceinline__ void dft_small<2, false>(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft_small<2, true>(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  // X[k] = sum_n x[n] (-+i)^{nk}
  float2 c0 = cadd(x0, x2), c1 = csub(x0, x2);
  float2 c2 = cadd(x1, x3), c3 = mul_rot<INV>(csub(x1, x3));
  x0 = cadd(c0, c2);
  x2 = csub(c0, c2);
  x1 = cadd(c1, c3);
  x3 = csub(c1, c3);
}

template <>
__device__ __forceinline__ void dft_small<4, false>(float2* v) { dft4<false>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void dft_small<4, true>(float2* v) { dft4<true>(v[0], v[1], v[2], v[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  // radix-2 split: even outputs from a[n] + a[n+4], odd outputs from
  // (a[n] - a[n+4]) W8^n, each through a 4-point DFT.
  const float h = 0.70710678118654752440f;  // 1/sqrt(2)
  float2 b0 = cadd(v[0], v[4]), b4 = csub(v[0], v[4]);
  float2 b1 = cadd(v[1], v[5]), b5 = csub(v[1], v[5]);
  float2 b2 = cadd(v[2], v[6]), b6 = csub(v[2], v[6]);
  float2 b3 = cadd(v[3], v[7]), b7 = csub(v[3], v[7]);
  // W8^1 = (1 -+ i)/sqrt2, W8^2 = -+i, W8^3 = (-1 -+ i)/sqrt2
  if (INV) {
    b5 = make_float2((b5.x - b5.y) * h, (b5.x + b5.y) * h);
    b6 = make_float2(-b6.y, b6.x);
    b7 = make_float2((-b7.x - b7.y) * h, (b7.x - b7.y) * h);
  } else {
    b5 = make_float2((b5.x + b5.y) * h, (b5.y - b5.x) * h);
    b6 = make_float2(b6.y, -b6.x);
    b7 = make_float2((b7.y - b7.x) * h, (-b7.x - b7.y) * h);
  }
  dft4<INV>(b0, b1, b2, b3);
  dft4<INV>(b4, b5, b6, b7);
  v[0] = b0; v[2] = b1; v[4] = b2; v[6] = b3;
  v[1] = b4; v[3] = b5; v[5] = b6; v[7] = b7;
}

template <>
__device__ __forceinline__ void dft_small<8, false>(float2* v) { dft8<false>(v); }
template <>
__device__ __forceinline__ void dft_small<8, true>(float2* v) { dft8<true>(v); }

template <int L>
struct FftTeam {
  static constexpr int TL = (L / 8 < 32) ? (L / 8) : 32;  // lanes per transform
  static constexpr int PER_WARP = 32 / TL;                 // transforms per warp
  static_assert(L >= 16 && (L & (L - 1)) == 0, "power-of-two length >= 16");
};

// One Stockham pass with radix R after NS points have been combined.
template <int L, int R, int NS, bool INV>
__device__ __forceinline__ void stockham_pass(float2* buf, const float2* __restrict__ tw, int lane, bool active) {
  constexpr int TL = FftTeam<L>::TL;
  constexpr int NB = L / R;
  constexpr int PER = NB / TL;
  static_assert(PER >= 1 && NB % TL == 0, "team too large for this pass");
  float2 v[PER][R];
  if (active) {
#pragma unroll
    for (int m = 0; m < PER; ++m) {
      const int j = lane + m * TL;
#pragma unroll
      for (int r = 0; r < R; ++r) v[m][r] = buf[j + r * NB];
      if (NS > 1) {
        const int jm = j & (NS - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(jm * r) * (L / (NS * R))];
          if (INV) w.y = -w.y;
          v[m][r] = cmul(v[m][r], w);
        }
      }
      dft_small<R, INV>(v[m]);
    }
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int m = 0; m < PER; ++m) {
      const int j = lane + m * TL;
      const int jm = j & (NS - 1);
      const int base = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[base + r * NS] = v[m][r];
    }
  }
  __syncwarp();
}

template <int L, int NS, bool INV>
__device__ __forceinline__ void fft_passes(float2* buf, const float2* __restrict__ tw, int lane, bool active) {
  if constexpr (NS < L) {
    constexpr int REM = L / NS;
    constexpr int R = (REM >= 8) ? 8 : REM;
    stockham_pass<L, R, NS, INV>(buf, tw, lane, active);
    fft_passes<L, NS * R, INV>(buf, tw, lane, active);
  }
}

// In-place length-L transform of buf[0..L) in shared memory by one team.
// Every lane of the warp must call this (inactive lanes pass active = false).
template <int L, bool INV>
__device__ __forceinline__ void team_fft(float2* buf, const float2* __restrict__ tw, int lane, bool active) {
  fft_passes<L, 1, INV>(buf, tw, lane, active);
}

}  // namespace elf
