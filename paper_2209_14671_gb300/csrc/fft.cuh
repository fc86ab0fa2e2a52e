// Device building blocks: complex arithmetic and a shared-memory FFT.
//
// A length-L transform, L = P * Q (P >= Q, powers of two), is owned by a team of
// Q lanes of one warp and done in two passes over its shared-memory buffer
// (the "four-step" split of the DFT index):
//   pass 1  lane l reads x[l + Q j] (j < P), does a P-point DFT in registers,
//           multiplies by W_L^{l k1} and writes the result transposed (k1-major);
//   pass 2  lane l takes rows k1 = l + Q m, does Q-point DFTs in registers and
//           writes X[k1 + P k2] in natural order.
// Buffers use the padded index p(i) = i + floor(i / Q) (one spare element after
// every Q), which makes the strided accesses of both passes bank-conflict free
// within each half-warp.  Twiddles W_L^{l k1} come from a table laid out
// [k1][l] (built in FP64 on the host), the constants of the in-register DFTs
// are exact values of cos(k pi / 16).  Transforms are unnormalised: forward
// X[k] = sum_x x[x] e^{-2 pi i k x / L}, inverse with e^{+2 pi i k x / L}.
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

// cos(k pi / 16), k = 0..8
__device__ __forceinline__ constexpr float cos16(int k) {
  return k == 0 ? 1.0f
       : k == 1 ? 0.98078528040323043058f
       : k == 2 ? 0.92387953251128673848f
       : k == 3 ? 0.83146961230254523567f
       : k == 4 ? 0.70710678118654757274f
       : k == 5 ? 0.55557023301960228867f
       : k == 6 ? 0.38268343236508983729f
       : k == 7 ? 0.19509032201612833135f
                : 0.0f;
}

// W_32^m = e^{-+2 pi i m / 32} for 0 <= m < 16 (sign by direction)
template <bool INV>
__device__ __forceinline__ float2 w32(int m) {
  const float c = (m <= 8) ? cos16(m) : -cos16(16 - m);
  const float s = (m <= 8) ? cos16(8 - m) : cos16(m - 8);  // sin(m pi / 16)
  return INV ? make_float2(c, s) : make_float2(c, -s);
}

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// o * W_32^m with the trivial factors (m = 0: 1, m = 8: -+i) resolved at compile time
template <bool INV>
__device__ __forceinline__ float2 twmul(float2 o, int m) {
  if (m == 0) return o;
  if (m == 8) return mul_rot<INV>(o);
  return cmul(o, w32<INV>(m));
}

// In-register DFT of M values (natural order in and out), radix-2 recursion
// with hand-written 2, 4 and 8-point kernels.
template <int M, bool INV>
struct Dft {
  static __device__ __forceinline__ void run(float2* v) {
    float2 e[M / 2], o[M / 2];
#pragma unroll
    for (int k = 0; k < M / 2; ++k) {
      e[k] = v[2 * k];
      o[k] = v[2 * k + 1];
    }
    Dft<M / 2, INV>::run(e);
    Dft<M / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < M / 2; ++k) {
      const float2 t = twmul<INV>(o[k], k * (32 / M));
      v[k] = cadd(e[k], t);
      v[k + M / 2] = csub(e[k], t);
    }
  }
};

template <bool INV>
struct Dft<1, INV> {
  static __device__ __forceinline__ void run(float2*) {}
};

template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 c0 = cadd(v[0], v[2]), c1 = csub(v[0], v[2]);
    const float2 c2 = cadd(v[1], v[3]), c3 = mul_rot<INV>(csub(v[1], v[3]));
    v[0] = cadd(c0, c2);
    v[2] = csub(c0, c2);
    v[1] = cadd(c1, c3);
    v[3] = csub(c1, c3);
  }
};

template <bool INV>
struct Dft<8, INV> {
  static __device__ __forceinline__ void run(float2* v) {
    // even outputs from a[n] + a[n+4], odd outputs from (a[n] - a[n+4]) W8^n
    const float h = cos16(4);
    float2 b[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      b[k] = cadd(v[k], v[k + 4]);
      b[k + 4] = csub(v[k], v[k + 4]);
    }
    if (INV) {
      b[5] = make_float2((b[5].x - b[5].y) * h, (b[5].x + b[5].y) * h);
      b[6] = make_float2(-b[6].y, b[6].x);
      b[7] = make_float2((-b[7].x - b[7].y) * h, (b[7].x - b[7].y) * h);
    } else {
      b[5] = make_float2((b[5].x + b[5].y) * h, (b[5].y - b[5].x) * h);
      b[6] = make_float2(b[6].y, -b[6].x);
      b[7] = make_float2((b[7].y - b[7].x) * h, (-b[7].x - b[7].y) * h);
    }
    Dft<4, INV>::run(b);
    Dft<4, INV>::run(b + 4);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = b[k];
      v[2 * k + 1] = b[k + 4];
    }
  }
};

template <int L>
struct FftTeam {
  static_assert(L >= 16 && L <= 1024 && (L & (L - 1)) == 0, "power-of-two length 16..1024");
  static constexpr int LOG = (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6 : (L == 128) ? 7 : (L == 256) ? 8
                           : (L == 512) ? 9 : 10;
  static constexpr int Q = 1 << (LOG / 2);        // lanes per transform
  static constexpr int P = L / Q;                 // values per lane (P >= Q)
  static constexpr int TL = Q;
  static constexpr int PER_WARP = 32 / Q;
  static constexpr int PADDED = L + L / Q;        // buffer length with padding
  static __device__ __forceinline__ int pidx(int i) { return i + (i >> (LOG / 2)); }
};

// Twiddle table of a team transform: tw[k1 * Q + l] = W_L^{l k1} (forward sign).
//
// The buffer of one transform holds element e at buf[e * S] (S = 1: contiguous; a
// larger S walks a column of a row-major array), e < PADDED; data index i lives at
// e = pidx(i).  Every lane of the warp must call these (inactive lanes pass
// active = false).
//
// team_fft_core: v[j] = x[lane + Q j] (j < P) on entry, the values pass 1 reads;
// on return v[m * Q + k2] = X[k1 + P k2] with k1 = lane + Q m.  buf is scratch.
template <int L, bool INV, int S = 1>
__device__ __forceinline__ void team_fft_core(float2* v, float2* buf, const float2* __restrict__ tw, int lane,
                                              bool active) {
  using T = FftTeam<L>;
  constexpr int P = T::P, Q = T::Q;
  if (active) {
    Dft<P, INV>::run(v);
#pragma unroll
    for (int k = 1; k < P; ++k) {
      float2 w = tw[k * Q + lane];
      if (INV) w.y = -w.y;
      v[k] = cmul(v[k], w);
    }
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int k = 0; k < P; ++k) buf[(k * (Q + 1) + lane) * S] = v[k];
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int m = 0; m < P / Q; ++m) {
      const int k1 = lane + Q * m;
#pragma unroll
      for (int l = 0; l < Q; ++l) v[m * Q + l] = buf[(k1 * (Q + 1) + l) * S];
      Dft<Q, INV>::run(v + m * Q);
    }
  }
  __syncwarp();
}

// team_fft_regs: team_fft_core, then X in natural order into buf (element pidx(k)).
template <int L, bool INV, int S = 1>
__device__ __forceinline__ void team_fft_regs(float2* v, float2* buf, const float2* __restrict__ tw, int lane,
                                              bool active) {
  using T = FftTeam<L>;
  constexpr int P = T::P, Q = T::Q;
  team_fft_core<L, INV, S>(v, buf, tw, lane, active);
  if (active) {
#pragma unroll
    for (int m = 0; m < P / Q; ++m) {
      const int k1 = lane + Q * m;
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) buf[T::pidx(k1 + P * k2) * S] = v[m * Q + k2];
    }
  }
  __syncwarp();
}

// team_fft: in-place transform of buf.  Inputs outside [lo, lo + cnt) are taken as
// zero without being read.
template <int L, bool INV, int S = 1>
__device__ __forceinline__ void team_fft(float2* buf, const float2* __restrict__ tw, int lane, bool active,
                                         int lo = 0, int cnt = L) {
  constexpr int P = FftTeam<L>::P, Q = FftTeam<L>::Q;
  float2 v[P];
  if (active) {
#pragma unroll
    for (int j = 0; j < P; ++j)
      v[j] = ((unsigned)(lane + Q * j - lo) < (unsigned)cnt) ? buf[(lane + (Q + 1) * j) * S]
                                                             : make_float2(0.f, 0.f);
  }
  team_fft_regs<L, INV, S>(v, buf, tw, lane, active);
}

}  // namespace elf
