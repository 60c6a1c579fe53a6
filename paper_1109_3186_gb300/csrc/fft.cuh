// fft.cuh -- register/shared-memory radix-16 Stockham FFT building blocks.
//
// An FFT of length L (power of two, 16 <= L <= 4096) is split into radix-16
// stages followed by at most one radix-2/4/8 stage.  Every thread holds
// exactly 16 complex values; thread jt of a sequence starts with elements
// jt + k L/16 (k = 0..15) and ends with the transformed elements at the same
// positions, so global loads and stores around the core are plain strided
// accesses that coalesce across the threads of a warp.  Values cross threads
// only through shared memory, one exchange between consecutive stages.
//
// Two shared-memory tile layouts serve the two passes of the large
// transforms:
//   ROWMAJOR = true : C sequences of length L stored one after the other;
//                     threads are numbered jt-fastest (rows of a matrix).
//   ROWMAJOR = false: C sequences interleaved element-major (columns of a
//                     matrix); threads are numbered sequence-fastest.
// Both pad one slot every 16 so that every stage is free of bank conflicts.
#pragma once
#include <cuda_runtime.h>

namespace chirp {

struct __align__(8) c32 {
  float x, y;
};

// Complex add and subtract as one paired FP32 instruction each (add/sub
// .rn.f32x2: both lanes rounded exactly like two scalar operations), which
// halves the butterflies' instruction count.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rc, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rc;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rc;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rc, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rc;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -j (forward) or +j (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mj(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// twiddle tables in global memory (filled once, FP64 rounded once to FP32):
//   tw_coarse[m] = exp(-2 pi j m / 4096)      m < 4096
//   tw_fine[m]   = exp(-2 pi j m / 2^24)      m < 4096
//   stage[o(Ns) + m] = (w, w^4), w = exp(-2 pi j m / (16 Ns)), m < Ns, for
//                  the radix-16 stages of span Ns = 16 (o = 0) and 256 (o = 16):
//                  the butterflies of a warp read consecutive 16-byte entries
//                  (the same factors taken from tw_coarse sit 128 bytes or more
//                  apart, one L1 wavefront per lane)
struct Twiddles {
  const float2* coarse;
  const float2* fine;
  const float4* stage;
};
constexpr int kStageTwiddles = 16 + 256;

// exp(-+2 pi j m / 4096), m in [0, 4096)
template <bool INV>
__device__ __forceinline__ float2 tw4096(const Twiddles& t, int m) {
  float2 w = __ldg(t.coarse + m);
  return INV ? cconj(w) : w;
}

// exp(-+2 pi j e / nfft) for e in [0, nfft), nfft = 2^log2n <= 2^24
template <bool INV>
__device__ __forceinline__ float2 tw_big(const Twiddles& t, unsigned e, int log2n) {
  unsigned e24 = e << (24 - log2n);
  float2 w = cmul(__ldg(t.coarse + (e24 >> 12)), __ldg(t.fine + (e24 & 4095u)));
  return INV ? cconj(w) : w;
}

// ---------------------------------------------------------------- small DFTs
// In place, natural order in and out, sign -1 (forward) or +1 (INV).
template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a0 = cadd(x0, x2), a1 = csub(x0, x2);
  float2 a2 = cadd(x1, x3), d = csub(x1, x3);
  x0 = cadd(a0, a2);
  x2 = csub(a0, a2);
  // x1 = a1 + (-+j) d, x3 = a1 - (-+j) d: the swapped lanes stay scalar
  if (INV) {
    x1 = make_float2(a1.x - d.y, a1.y + d.x);
    x3 = make_float2(a1.x + d.y, a1.y - d.x);
  } else {
    x1 = make_float2(a1.x + d.y, a1.y - d.x);
    x3 = make_float2(a1.x - d.y, a1.y + d.x);
  }
}

template <bool INV>
__device__ __forceinline__ float2 rot8(float2 a, int m) {  // a * exp(-+2 pi j m / 8), m = 0..3
  const float r = 0.70710678118654752440f;
  switch (m & 7) {
    case 0: return a;
    case 1: return INV ? make_float2(r * (a.x - a.y), r * (a.x + a.y)) : make_float2(r * (a.x + a.y), r * (a.y - a.x));
    case 2: return mul_mj<INV>(a);
    default: return INV ? make_float2(-r * (a.x + a.y), r * (a.x - a.y)) : make_float2(r * (a.y - a.x), -r * (a.x + a.y));
  }
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  // 8 = 2 x 4: n = 4 n1 + n2 ... written as: DFT4 over n1 of x[2 n1 + n2], twiddle, DFT2
  dft4<INV>(v[0], v[2], v[4], v[6]);
  dft4<INV>(v[1], v[3], v[5], v[7]);
  // A[k1][n2] at v[2 k1 + n2]; multiply by W8^(n2 k1)
  v[3] = rot8<INV>(v[3], 1);
  v[5] = rot8<INV>(v[5], 2);
  v[7] = rot8<INV>(v[7], 3);
  dft2<INV>(v[0], v[1]);
  dft2<INV>(v[2], v[3]);
  dft2<INV>(v[4], v[5]);
  dft2<INV>(v[6], v[7]);
  // X[k1 + 4 k2] sits at v[2 k1 + k2]
  float2 t[8];
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
    for (int k2 = 0; k2 < 2; k2++) t[k1 + 4 * k2] = v[2 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = t[i];
}

template <bool INV>
__device__ __forceinline__ float2 rot16(float2 a, int m) {  // a * exp(-+2 pi j m / 16)
  const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
  const float r = 0.70710678118654752440f;
  float c, s;  // exp(-2 pi j m/16) = c - j s (forward)
  switch (m) {
    case 0: return a;
    case 1: c = c1; s = s1; break;
    case 2: c = r; s = r; break;
    case 3: c = s1; s = c1; break;
    case 4: return mul_mj<INV>(a);
    case 6: c = -r; s = r; break;
    case 9: c = -c1; s = -s1; break;
    default: c = 1.f; s = 0.f; break;  // not used
  }
  if (INV) s = -s;
  return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  // 16 = 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddle W16^(n2 k1), DFT4 over n2
#pragma unroll
  for (int n2 = 0; n2 < 4; n2++) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
#pragma unroll
  for (int k1 = 1; k1 < 4; k1++)
#pragma unroll
    for (int n2 = 1; n2 < 4; n2++) v[4 * k1 + n2] = rot16<INV>(v[4 * k1 + n2], n2 * k1);
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; k1++)
#pragma unroll
    for (int k2 = 0; k2 < 4; k2++) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = t[i];
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
  else dft16<INV>(v);
}

// ---------------------------------------------------------------- the core
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

// padded shared-memory slot of linear index i (one pad slot every 16)
__device__ __forceinline__ int padidx(int i) { return i + (i >> 4); }

template <int L, int C>
struct FftTile {
  static constexpr int T = L / 16;                   // threads per sequence
  static constexpr int THREADS = T * C;
  static constexpr int SLOTS = (L * C) + (L * C) / 16;  // padded float2 count
};

// Shared-memory index of element i of sequence s.
template <int L, int C, bool ROWMAJOR>
__device__ __forceinline__ int tile_idx(int i, int s) {
  return padidx(ROWMAJOR ? s * L + i : i * C + s);
}

// v[k] *= a w1^k for k = 0..15, given w1 and w4 = w1^4 (exact table values).
// Powers are formed on the fly as (a w4^b) w1^q with k = 4b + q, so every
// factor is at most a few products away from a table value (a running product
// would add one rounding per step) and only a handful of registers are live.
__device__ __forceinline__ void apply_pow16(float2 (&v)[16], float2 a, float2 w1, float2 w4) {
  const float2 w2 = cmul(w1, w1);
  const float2 w3 = cmul(w2, w1);
  float2 base = a;
#pragma unroll
  for (int b = 0; b < 4; b++) {
    v[4 * b] = cmul(v[4 * b], base);
    v[4 * b + 1] = cmul(v[4 * b + 1], cmul(base, w1));
    v[4 * b + 2] = cmul(v[4 * b + 2], cmul(base, w2));
    v[4 * b + 3] = cmul(v[4 * b + 3], cmul(base, w3));
    if (b < 3) base = cmul(base, w4);
  }
}

// The same for a = 1: v[0] is left alone and the first row of powers is
// w1, w2, w3 themselves (the products with an exact 1 are skipped).
__device__ __forceinline__ void apply_pow16_unit(float2 (&v)[16], float2 w1, float2 w4) {
  const float2 w2 = cmul(w1, w1);
  const float2 w3 = cmul(w2, w1);
  v[1] = cmul(v[1], w1);
  v[2] = cmul(v[2], w2);
  v[3] = cmul(v[3], w3);
  float2 base = w4;
#pragma unroll
  for (int b = 1; b < 4; b++) {
    v[4 * b] = cmul(v[4 * b], base);
    v[4 * b + 1] = cmul(v[4 * b + 1], cmul(base, w1));
    v[4 * b + 2] = cmul(v[4 * b + 2], cmul(base, w2));
    v[4 * b + 3] = cmul(v[4 * b + 3], cmul(base, w3));
    if (b < 3) base = cmul(base, w4);
  }
}

// Stockham stage helpers -------------------------------------------------
// One radix-R stage of span Ns over L points for butterfly j:
//   in:  a[j + q L/R],  twiddle W_{Ns R}^{q (j mod Ns)},  DFT_R,
//   out: b[(j / Ns) Ns R + (j mod Ns) + q Ns].
template <int L, int R, bool INV>
__device__ __forceinline__ void stage_twiddle(float2* v, int j, int Ns, const Twiddles& tw) {
  if (Ns == 1) return;
  int jm = j & (Ns - 1);
  int scale = 4096 / (Ns * R);
  if constexpr (R == 16) {
    // radix-16 stages have Ns = 16 or 256 (L <= 4096)
    float2 (&vv)[16] = *reinterpret_cast<float2(*)[16]>(v);
    const float4 t = __ldg(tw.stage + (Ns == 16 ? 0 : 16) + jm);
    float2 w1 = make_float2(t.x, t.y), w4 = make_float2(t.z, t.w);
    if (INV) {
      w1 = cconj(w1);
      w4 = cconj(w4);
    }
    apply_pow16_unit(vv, w1, w4);
  } else {
#pragma unroll
    for (int q = 1; q < R; q++) v[q] = cmul(v[q], tw4096<INV>(tw, (q * jm * scale) & 4095));
  }
}

// v[k] *= W_N^(-+ m (j0 + k T)) for k = 0..15 (N = 2^log2n), from three
// table look-ups per thread instead of two per element.
template <bool INV>
__device__ __forceinline__ void twiddle_run(float2 (&v)[16], unsigned m, unsigned j0, unsigned T,
                                            int log2n, const Twiddles& tw) {
  const unsigned mask = (1u << log2n) - 1u;
  apply_pow16(v, tw_big<INV>(tw, (m * j0) & mask, log2n), tw_big<INV>(tw, (m * T) & mask, log2n),
              tw_big<INV>(tw, (4u * m * T) & mask, log2n));
}

// The same with the per-thread factor W_N^(m j0) given as base (forward
// sign, e.g. from a per-row table read with consecutive addresses): the two
// remaining look-ups are uniform across the threads of a row.
template <bool INV>
__device__ __forceinline__ void twiddle_run_base(float2 (&v)[16], float2 base, unsigned m,
                                                 unsigned T, int log2n, const Twiddles& tw) {
  const unsigned mask = (1u << log2n) - 1u;
  apply_pow16(v, INV ? cconj(base) : base, tw_big<INV>(tw, (m * T) & mask, log2n),
              tw_big<INV>(tw, (4u * m * T) & mask, log2n));
}

// Thread -> (column s, butterfly jt) of a column pass (ROWMAJOR = false).
// For the 512-point transform (C = 8 columns of T = 32 threads) lane bit 4
// carries bit 4 of jt, so that threads jt and jt ^ 16 share a warp: between
// the last radix-16 stage and the radix-2 stage they are the only threads
// that trade values, which fft_core<..., XSHFL = true> then does by warp
// shuffles instead of a shared-memory round trip.  A warp still covers 8
// consecutive columns of 4 rows, as in the plain order s = tid % C.
template <int L, int C>
constexpr bool kColShfl = (L == 512 && C == 8);

template <int L, int C>
__device__ __forceinline__ void col_thread(int tid, int& s, int& jt) {
  if constexpr (kColShfl<L, C>) {
    s = tid & 7;
    jt = ((tid >> 3) & 1) | (((tid >> 5) & 7) << 1) | (((tid >> 4) & 1) << 4);
  } else {
    s = tid % C;
    jt = tid / C;
  }
}

// Forward (INV=false) or inverse (INV=true, unnormalised) FFT of length L.
// On entry v[k] = element jt + k L/16 of sequence s; on exit the same
// positions hold the transform.  sm: at least FftTile<L,C>::SLOTS float2.
// All threads of the block that own (s, jt) pairs must call it together.
// XSHFL (512 points, threads placed by col_thread): the exchange before the
// radix-2 stage by warp shuffles; every lane of each warp must take part.
template <int L, int C, bool ROWMAJOR, bool INV, bool XSHFL = false>
__device__ __forceinline__ void fft_core(float2 (&v)[16], float2* sm, int s, int jt,
                                         const Twiddles& tw) {
  static_assert(L >= 16 && L <= 4096 && (L & (L - 1)) == 0, "L");
  constexpr int LOG = ilog2c(L);
  constexpr int N16 = LOG / 4;           // radix-16 stages
  constexpr int RLAST = 1 << (LOG % 4);  // trailing radix (1 = none)
  constexpr int T = L / 16;
  static_assert(!XSHFL || (L == 512 && C == 8 && !ROWMAJOR), "XSHFL: 512-point column pass");

  int Ns = 1;
#pragma unroll
  for (int st = 0; st < N16; st++) {
    // radix-16 stage: butterfly j = jt reads a[jt + q T] (already in v)
    stage_twiddle<L, 16, INV>(v, jt, Ns, tw);
    dft_r<16, INV>(v);
    if constexpr (XSHFL) {
      if (st == N16 - 1) {
        // v[q] is element 256 h + (jt & 15) + 16 q (h = bit 4 of jt); the
        // radix-2 stage wants elements jt + 32 k, k < 16: the even q of
        // thread (jt & 15) and then of thread (jt & 15) + 16 for h = 0, their
        // odd q for h = 1.  Each thread keeps its own half and trades the
        // other half with its partner jt ^ 16 (lane ^ 16).
        const bool h = (jt >> 4) & 1;
        float2 got[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const float2 val = h ? v[2 * i] : v[2 * i + 1];
          got[i].x = __shfl_xor_sync(0xffffffffu, val.x, 16);
          got[i].y = __shfl_xor_sync(0xffffffffu, val.y, 16);
        }
        float2 nv[16];
#pragma unroll
        for (int k = 0; k < 8; k++) {
          nv[k] = h ? got[k] : v[2 * k];
          nv[8 + k] = h ? v[2 * k + 1] : got[k];
        }
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = nv[k];
        break;  // on to the radix-2 stage
      }
    }
    const bool last = (st == N16 - 1) && (RLAST == 1);
    if (last) return;  // outputs b[jt + q T] == positions already held
    // write b[(j/Ns) Ns 16 + j%Ns + q Ns], then read the next stage inputs
    {
      int base = (jt / Ns) * Ns * 16 + (jt & (Ns - 1));
#pragma unroll
      for (int q = 0; q < 16; q++) sm[tile_idx<L, C, ROWMAJOR>(base + q * Ns, s)] = v[q];
    }
    __syncthreads();
    Ns *= 16;
    if (st + 1 < N16) {
#pragma unroll
      for (int q = 0; q < 16; q++) v[q] = sm[tile_idx<L, C, ROWMAJOR>(jt + q * T, s)];
    } else {
      // trailing radix-RLAST stage: butterflies j = jt + u T, u < 16/RLAST,
      // each reads a[j + q L/RLAST]; element index = jt + (u + q 16/RLAST) T
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = sm[tile_idx<L, C, ROWMAJOR>(jt + k * T, s)];
    }
    __syncthreads();
  }
  if constexpr (RLAST > 1) {
    constexpr int U = 16 / RLAST;
    // Ns == L / RLAST here.  v[u + q U] holds a[jt + u T + q L/RLAST].
#pragma unroll
    for (int u = 0; u < U; u++) {
      float2 w[RLAST];
#pragma unroll
      for (int q = 0; q < RLAST; q++) w[q] = v[u + q * U];
      const int j = jt + u * T;
      if constexpr (N16 > 0) stage_twiddle<L, RLAST, INV>(w, j, L / RLAST, tw);
      dft_r<RLAST, INV>(w);
      // output b[j + q Ns] = element jt + (u + q U) T  -> same register slot
#pragma unroll
      for (int q = 0; q < RLAST; q++) v[u + q * U] = w[q];
    }
  }
}

}  // namespace chirp
