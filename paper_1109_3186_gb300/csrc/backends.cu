// backends.cu -- CUDA-core back-ends that consume dedispersed voltages.
//
// Chirpolator (correlate): per dump m the zero-lag products
//   V_pq = sum_{t in dump} y_p(t) y_q(t)^*   (p <= q, autos included),
// the pair mixing x_pq = s_p s_q^* of Eq. xpq integrated and dumped.
// Chimageator, plain FP32 form: per dump and pixel
//   P = sum_{t in dump} |sum_a W_pa y_a(t)|^2
// (direct beamforming, Sec. 2.4.2, detected and integrated).
//
// Both accumulate in FP32 with a two-level sum (a short inner run, then the
// running total) so that a 4096-sample dump stays within the 1e-5 relative
// budget of the FP32 path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace chirp {

// ------------------------------------------------------------------ correlate
// The M x M product is cut into 4 x 4 antenna tiles on or above the diagonal.
// One warp owns one tile of one dump: lane l takes the samples l, l + 32, ...
// of the dump, keeps the tile's products in registers, and the 32 lane
// partials are summed with warp shuffles at the end.
//
// Up to 16 antennas (NT = ceil(M/4) <= 4 tile rows, at most 10 tiles) one CTA
// holds every tile of a dump and streams the dump through shared memory
// (k_correlate_staged): chunks of kCorrChunk samples of every antenna row are
// fetched with cp.async (16-byte copies when rows and dumps start on 16-byte
// boundaries) into two buffers, the next chunk in flight while the warps
// multiply the current one.  Rows M .. 4 NT - 1 stay zero, and a dump's ragged
// last chunk is zero-filled, so the inner loop has no bounds or predicates.
// Each complex product-accumulate u_a conj(w_b) is two paired FP32 FMAs on
// lane-split accumulators (fma.rn.f32x2):
//   P += (u.re w.re, u.im w.im),  Q += (u.im w.re, u.re w.im),
//   Re V = P.lo + P.hi,  Im V = Q.lo - Q.hi,
// so a sample needs its (re, im) pair and one swapped copy (im, re) per row
// antenna, and no broadcasts or sign flips.  Diagonal tiles form only their
// upper triangle.  Above 16 antennas the antennas form blocks of 12: one
// launch takes each block alone (its upper tiles), a second each pair of
// blocks, staging both blocks' rows.
constexpr int kCorrTile = 4;
constexpr int kCorrChunk = 256;
constexpr int kCorrStagedMaxAnt = 16;

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(float2* smem, const float2* gmem) { cp_async8(smem, gmem); }
__device__ __forceinline__ void cp_async_elem(__nv_bfloat162* smem, const __nv_bfloat162* gmem) {
  cp_async4(smem, gmem);
}
__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fma2(unsigned long long& acc, unsigned long long a,
                                     unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
// A staged sample as the (re, im) pair and, with SW, also the (im, re) pair.
template <bool SW>
__device__ __forceinline__ void sample_pair(const float2* p, unsigned long long& v,
                                            unsigned long long& vs) {
  v = *reinterpret_cast<const unsigned long long*>(p);
  if (SW) {
    const float2 a = unpack2(v);
    vs = pack2(a.y, a.x);
  }
}
template <bool SW>
__device__ __forceinline__ void sample_pair(const __nv_bfloat162* p, unsigned long long& v,
                                            unsigned long long& vs) {
  // BF16 -> FP32 is exact: the 16 bits become the top half of the float
  const unsigned b = *reinterpret_cast<const unsigned*>(p);
  const float re = __uint_as_float(b << 16), im = __uint_as_float(b & 0xffff0000u);
  v = pack2(re, im);
  if (SW) vs = pack2(im, re);
}
__device__ __forceinline__ void zero_elem(float2* p) { *p = make_float2(0.f, 0.f); }
__device__ __forceinline__ void zero_elem(__nv_bfloat162* p) {
  *reinterpret_cast<unsigned*>(p) = 0u;
}

// 96 registers: two CTAs of 10 warps (NT = 4) or three of 6 (NT = 3) per SM
// (single-warp CTAs, NT = 1, are limited by shared memory instead: 128).
// Antennas form blocks of BA = 4 NT.  PAIR = false: CTA (dump, I) takes block
// I alone -- its NT (NT + 1) / 2 upper 4 x 4 tiles, one per warp (up to 16
// antennas this is the whole product).  PAIR = true: CTA (dump, (I, J)),
// I < J (the task index runs over the strict upper triangle of blocks),
// stages block I's rows, then block J's, and its NT x NT warps each own one
// 4 x 4 tile of the pairs (block I antenna, block J antenna).
// task_fast: the task (block or block pair) is grid dimension x and the dump
// y, so that the CTAs of one dump run together and the block pairs that share
// a block find its rows in L2; otherwise the dump is x and the task y.
struct CorrBatch {
  CorrJob job[kCorrBatchMax];
};

template <typename T, int NT, bool VEC16, bool PAIR>
__global__ void __maxnreg__(NT == 1 ? 128 : 96)
    k_correlate_staged(const __grid_constant__ CorrBatch batch, long long n_samp, int M, int L,
                       int task_fast) {
  // this CTA's DM (grid dimension z), dump and task
  const CorrJob& job = batch.job[blockIdx.z];
  const unsigned dump_i = task_fast ? blockIdx.y : blockIdx.x;
  const unsigned task = task_fast ? blockIdx.x : blockIdx.y;
  if (dump_i >= job.n_m) return;
  const T* __restrict__ y = static_cast<const T*>(job.y);
  float2* __restrict__ vis = job.vis;
  const int* __restrict__ dump_list = job.dump_list;
  const long long m_base = job.m_base, first = job.first, last = job.last;
  constexpr int BA = kCorrTile * NT;  // antennas of a block
  constexpr int NTH = PAIR ? 32 * NT * NT : 32 * NT * (NT + 1) / 2;
  constexpr int ROWS = PAIR ? 2 * BA : BA;  // stage rows, zero-padded
  constexpr int CH = kCorrChunk;
  constexpr int STAGE = ROWS * CH;
  extern __shared__ __align__(16) unsigned char ring_raw[];
  T* ring = reinterpret_cast<T*>(ring_raw);  // [2][ROWS][CH]
  const long long m = dump_list ? (long long)dump_list[dump_i] : m_base + dump_i;
  const int n_pair = M * (M + 1) / 2;
  float2* out = vis + m * n_pair;
  if (m < first || m > last) {
    if (!PAIR && task == 0)
      for (int i = threadIdx.x; i < n_pair; i += NTH) out[i] = make_float2(0.f, 0.f);
    return;
  }
  int I = (int)task, J = I;
  if (PAIR) {  // strict upper triangle of SB x SB blocks, row-major
    const int SB = (M + BA - 1) / BA;
    int rem = (int)task;
    I = 0;
    while (rem >= SB - 1 - I) {
      rem -= SB - 1 - I;
      I++;
    }
    J = I + 1 + rem;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  int ti = 0, tj;
  if (PAIR) {
    ti = warp / NT;
    tj = warp % NT;
  } else {  // one upper tile of the block per warp
    int rem = warp;
    while (rem >= NT - ti) {
      rem -= NT - ti;
      ti++;
    }
    tj = ti + rem;
  }
  const bool diag = !PAIR && ti == tj;
  // stage rows [0, nA): antennas I BA + r; [BA, BA + nB): antennas J BA + r
  const int nA = min(BA, M - I * BA);
  const int nB = PAIR ? min(BA, M - J * BA) : 0;
  const int zA = BA - nA, zB = PAIR ? BA - nB : 0;  // padded rows stay zero
  for (int i = threadIdx.x; i < 2 * (zA + zB) * CH; i += NTH) {
    const int st = i / ((zA + zB) * CH), k = i % ((zA + zB) * CH);
    const int r = k / CH;
    zero_elem(ring + st * STAGE + (r < zA ? nA + r : BA + nB + (r - zA)) * CH + k % CH);
  }
  // sample 0 of the dump: antenna I BA (block I) and antenna J BA (block J)
  const T* srcA = y + (long long)I * BA * n_samp + m * L;
  const T* srcB = y + (long long)J * BA * n_samp + m * L;
  const int n_rows = nA + nB;
  const int n_chunks = (L + CH - 1) / CH;
  auto fetch = [&](int c) {
    if (c < n_chunks) {
      T* buf = ring + (c & 1) * STAGE;
      const int t0 = c * CH, len = min(CH, L - t0);
      if constexpr (VEC16) {  // rows, dumps and len are multiples of EPV samples
        constexpr int EPV = 16 / (int)sizeof(T);
        constexpr int U = CH / EPV;
        for (int e = threadIdx.x; e < n_rows * U; e += NTH) {
          const int r = e / U, i = EPV * (e % U);
          const bool inA = !PAIR || r < nA;
          const T* s_row = inA ? srcA + (long long)r * n_samp : srcB + (long long)(r - nA) * n_samp;
          T* dst = buf + (inA ? r : BA + (r - nA)) * CH + i;
          if (i < len)
            cp_async16(dst, s_row + t0 + i);
          else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
      } else {
        for (int e = threadIdx.x; e < n_rows * CH; e += NTH) {
          const int r = e / CH, i = e % CH;
          const bool inA = !PAIR || r < nA;
          const T* s_row = inA ? srcA + (long long)r * n_samp : srcB + (long long)(r - nA) * n_samp;
          T* dst = buf + (inA ? r : BA + (r - nA)) * CH + i;
          if (i < len)
            cp_async_elem(dst, s_row + t0 + i);
          else
            zero_elem(dst);
        }
      }
    }
    cp_async_commit();  // possibly empty: keeps the group count in step
  };
  unsigned long long P[kCorrTile][kCorrTile], Q[kCorrTile][kCorrTile];
#pragma unroll
  for (int a = 0; a < kCorrTile; a++)
#pragma unroll
    for (int b = 0; b < kCorrTile; b++) P[a][b] = Q[a][b] = 0ull;
  fetch(0);
  for (int c = 0; c < n_chunks; c++) {
    cp_async_wait<0>();
    __syncthreads();  // chunk c is in; every warp is done with chunk c - 1
    fetch(c + 1);
    const T* buf = ring + (c & 1) * STAGE;
    const T* ri = buf + ti * kCorrTile * CH + lane;
    const T* rj = buf + ((PAIR ? BA : 0) + tj * kCorrTile) * CH + lane;
#pragma unroll 1
    for (int t = 0; t < CH; t += 32) {
      unsigned long long u[kCorrTile], us[kCorrTile];
#pragma unroll
      for (int a = 0; a < kCorrTile; a++) sample_pair<true>(ri + a * CH + t, u[a], us[a]);
      if (diag) {
#pragma unroll
        for (int b = 0; b < kCorrTile; b++)
#pragma unroll
          for (int a = 0; a <= b; a++) {
            fma2(P[a][b], u[a], u[b]);
            fma2(Q[a][b], us[a], u[b]);
          }
      } else {
#pragma unroll
        for (int b = 0; b < kCorrTile; b++) {
          unsigned long long w, unused;
          sample_pair<false>(rj + b * CH + t, w, unused);
#pragma unroll
          for (int a = 0; a < kCorrTile; a++) {
            fma2(P[a][b], u[a], w);
            fma2(Q[a][b], us[a], w);
          }
        }
      }
    }
  }
  cp_async_wait<0>();
  // lane a*4+b writes pair (p, q) = (I BA + ti*4+a, J BA + tj*4+b) if p <= q
  float2 mine = make_float2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < kCorrTile; a++)
#pragma unroll
    for (int b = 0; b < kCorrTile; b++) {
      const float2 pp = unpack2(P[a][b]), qq = unpack2(Q[a][b]);
      float2 v = make_float2(pp.x + pp.y, qq.x - qq.y);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (lane == a * kCorrTile + b) mine = v;
    }
  if (lane < kCorrTile * kCorrTile) {
    const int a = lane / kCorrTile, b = lane % kCorrTile;
    const int p = I * BA + ti * kCorrTile + a, q = J * BA + tj * kCorrTile + b;
    if (p < M && q < M && p <= q) out[p * M - p * (p - 1) / 2 + (q - p)] = mine;
  }
}

template <typename T, int NT, bool VEC16, bool PAIR>
static cudaError_t launch_staged(const CorrBatch& b, int n_jobs, long long max_m, long long n_samp,
                                 int n_ant, int dump_len, cudaStream_t st) {
  constexpr int BA = kCorrTile * NT;
  const size_t smem = (size_t)2 * (PAIR ? 2 : 1) * BA * kCorrChunk * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_correlate_staged<T, NT, VEC16, PAIR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long SB = (n_ant + BA - 1) / BA;
  const long long n_y = PAIR ? SB * (SB - 1) / 2 : SB;
  if (n_y < 1) return cudaSuccess;
  if (n_y > 65535) return cudaErrorInvalidConfiguration;
  const int task_fast = n_y > 1 && max_m <= 65535;
  const dim3 grid = task_fast ? dim3((unsigned)n_y, (unsigned)max_m, (unsigned)n_jobs)
                              : dim3((unsigned)max_m, (unsigned)n_y, (unsigned)n_jobs);
  k_correlate_staged<T, NT, VEC16, PAIR>
      <<<grid, PAIR ? 32 * NT * NT : 32 * NT * (NT + 1) / 2, smem, st>>>(b, n_samp, n_ant,
                                                                        dump_len, task_fast);
  return cudaGetLastError();
}

template <typename T, bool VEC16>
static cudaError_t launch_staged_nt(const CorrBatch& b, int n_jobs, long long max_m,
                                    long long n_samp, int n_ant, int dump_len, cudaStream_t st) {
#define CHIRP_CORR_ARGS b, n_jobs, max_m, n_samp, n_ant, dump_len, st
  switch (n_ant > kCorrStagedMaxAnt ? 0 : (n_ant + kCorrTile - 1) / kCorrTile) {
    case 0: {  // blocks of 12 antennas: the diagonal blocks, then the block pairs
      cudaError_t e = launch_staged<T, 3, VEC16, false>(CHIRP_CORR_ARGS);
      return e != cudaSuccess ? e : launch_staged<T, 3, VEC16, true>(CHIRP_CORR_ARGS);
    }
    case 1: return launch_staged<T, 1, VEC16, false>(CHIRP_CORR_ARGS);
    case 2: return launch_staged<T, 2, VEC16, false>(CHIRP_CORR_ARGS);
    case 3: return launch_staged<T, 3, VEC16, false>(CHIRP_CORR_ARGS);
    case 4: return launch_staged<T, 4, VEC16, false>(CHIRP_CORR_ARGS);
    default: return cudaErrorInvalidValue;
  }
#undef CHIRP_CORR_ARGS
}

template <typename T>
static cudaError_t correlate_batch(const CorrJob* jobs, int n_jobs, long long n_samp, int n_ant,
                                   int dump_len, cudaStream_t st) {
  if (n_jobs < 1 || n_jobs > kCorrBatchMax) return cudaErrorInvalidValue;
  CorrBatch b{};
  long long max_m = 0;
  // 16-byte copies when every row and dump starts on a 16-byte boundary of
  // 16-byte aligned arrays
  constexpr int EPV = 16 / (int)sizeof(T);
  bool vec16 = n_samp % EPV == 0 && dump_len % EPV == 0;
  for (int i = 0; i < n_jobs; i++) {
    b.job[i] = jobs[i];
    if (jobs[i].n_m < 0 || jobs[i].n_m >= (1LL << 31)) return cudaErrorInvalidConfiguration;
    max_m = std::max(max_m, jobs[i].n_m);
    vec16 = vec16 && ((uintptr_t)jobs[i].y & 15) == 0;
  }
  if (max_m <= 0) return cudaSuccess;
  if (vec16) return launch_staged_nt<T, true>(b, n_jobs, max_m, n_samp, n_ant, dump_len, st);
  return launch_staged_nt<T, false>(b, n_jobs, max_m, n_samp, n_ant, dump_len, st);
}

cudaError_t launch_correlate_batch(const CorrJob* jobs, int n_jobs, bool bf16, long long n_samp,
                                   int n_ant, int dump_len, cudaStream_t st) {
  return bf16 ? correlate_batch<__nv_bfloat162>(jobs, n_jobs, n_samp, n_ant, dump_len, st)
              : correlate_batch<float2>(jobs, n_jobs, n_samp, n_ant, dump_len, st);
}

cudaError_t launch_correlate(const float2* y, long long n_samp, int n_ant, int dump_len,
                             long long m_base, long long n_m, long long first, long long last,
                             float2* vis, cudaStream_t st, const int* dump_list) {
  const CorrJob j{y, vis, m_base, n_m, first, last, dump_list};
  return correlate_batch<float2>(&j, 1, n_samp, n_ant, dump_len, st);
}

cudaError_t launch_correlate_bf16(const void* y16, long long n_samp, int n_ant, int dump_len,
                                  long long m_base, long long n_m, long long first, long long last,
                                  float2* vis, cudaStream_t st, const int* dump_list) {
  const CorrJob j{y16, vis, m_base, n_m, first, last, dump_list};
  return correlate_batch<__nv_bfloat162>(&j, 1, n_samp, n_ant, dump_len, st);
}

// ------------------------------------------------------------------ beams from visibilities
// Exact identity: sum_t |sum_a W_pa y_a(t)|^2 = sum_{a,b} W_pa W_pb^* V_ab with
// V_ab = sum_t y_a y_b^* (the correlator's output), i.e. for the packed upper
// triangle  P_p = sum_{a<=b} Re(w_p,ab V_ab),  w_p,ab = c_ab W_pa W_pb^*,
// c = 1 on the diagonal, 2 above it.  In real form this is one FP32 GEMM per
// DM:  P[m][p] = sum_{k < 2 n_pair} V[m][k] B[k][p]  with V read as floats
// (re, im interleaved) and B[2 i][p] = Re w_p,i, B[2 i + 1][p] = -Im w_p,i
// (plan-time layout, rows padded to kVisBK, columns to kVisBN, zero-filled).
// Register-tiled SGEMM: a CTA computes 64 dumps x 128 pixels, each thread
// 4 dumps x 8 pixels, K in steps of 16 staged through double-buffered shared
// memory; FP32 products accumulated in k order.
constexpr int kVisBM = 64;
constexpr int kVisBN = 128;
constexpr int kVisBK = 16;

struct VisBatch {
  VisJob job[kCorrBatchMax];
};

// One 64-dump x 128-pixel tile: row tile bx of DM job bz, pixel tile by.
__device__ __forceinline__ void vis_tile(const VisBatch& batch, int K, const float* __restrict__ B,
                                         int ldb, int n_pix, long long bx, int by, int bz,
                                         float (&As)[2][kVisBK][kVisBM],
                                         float (&Bs)[2][kVisBK][kVisBN]) {
  const VisJob& job = batch.job[bz];
  const long long row0 = bx * kVisBM;
  if (row0 >= job.n_rows) return;
  const float* __restrict__ V = reinterpret_cast<const float*>(job.V);
  float* __restrict__ pow = job.pow;
  const int* __restrict__ dump_list = job.dump_list;
  const long long first = job.first, n_rows = job.n_rows;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int p0 = by * kVisBN;
  // loader coordinates: A 64 rows x 16 k (4 k per thread), B 16 k x 128 (8 per thread)
  const int a_row = tid / 4, a_k = (tid % 4) * 4;
  const long long ar = row0 + a_row;
  const float* a_src = nullptr;
  if (ar < n_rows) {
    const long long m = dump_list ? (long long)dump_list[ar] : first + ar;
    a_src = V + m * K;
  }
  const int b_k = tid / 16, b_c = (tid % 16) * 8;
  const float* b_src = B + (long long)b_k * ldb + p0 + b_c;
  const int n_kt = (K + kVisBK - 1) / kVisBK;
  float ra[4];
  float4 rb0, rb1;
  auto load = [&](int kt) {
    const int k0 = kt * kVisBK;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int k = k0 + a_k + j;
      ra[j] = (a_src && k < K) ? __ldg(a_src + k) : 0.f;
    }
    const float4* bp = reinterpret_cast<const float4*>(b_src + (long long)k0 * ldb);
    rb0 = __ldg(bp);
    rb1 = __ldg(bp + 1);
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int j = 0; j < 4; j++) As[buf][a_k + j][a_row] = ra[j];
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c]) = rb0;
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c + 4]) = rb1;
  };
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[i][j] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < n_kt; kt++) {
    const int cur = kt & 1;
    if (kt + 1 < n_kt) load(kt + 1);
#pragma unroll
    for (int k = 0; k < kVisBK; k++) {
      const float4 a = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < n_kt) {
      store(cur ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const long long r = row0 + ty * 4 + i;
    if (r >= n_rows) continue;
    const long long m = dump_list ? (long long)dump_list[r] : first + r;
    float* out = pow + m * n_pix;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int p = p0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (p < n_pix) out[p] = acc[i][j];
    }
  }
}

// The tiles of a virtual grid of vx row tiles x vy pixel tiles x vz DMs, row
// tile fastest; a CTA takes tiles vb = blockIdx.x, + gridDim.x, ... (one each
// when the grid covers them all, fewer CTAs when it runs beside other work).
__global__ void __launch_bounds__(256) k_beam_from_vis(const __grid_constant__ VisBatch batch,
                                                       int K, const float* __restrict__ B,
                                                       int ldb, int n_pix, long long vx, int vy,
                                                       int vz) {
  __shared__ __align__(16) float As[2][kVisBK][kVisBM];
  __shared__ __align__(16) float Bs[2][kVisBK][kVisBN];
  const long long n_tiles = vx * vy * vz;
  for (long long vb = blockIdx.x; vb < n_tiles; vb += gridDim.x) {
    if (vb != blockIdx.x) __syncthreads();  // the previous tile's reads of As / Bs are done
    vis_tile(batch, K, B, ldb, n_pix, vb % vx, (int)((vb / vx) % vy), (int)(vb / (vx * vy)), As,
             Bs);
  }
}

int beam_vis_rows(int n_ant) { return ((n_ant * (n_ant + 1) + kVisBK - 1) / kVisBK) * kVisBK; }
int beam_vis_ld(int n_pix) { return ((n_pix + kVisBN - 1) / kVisBN) * kVisBN; }

cudaError_t launch_beam_from_vis_batch(const VisJob* jobs, int n_jobs, const float* wvis,
                                       int n_ant, int n_pix, cudaStream_t st, int max_ctas) {
  if (n_jobs < 1 || n_jobs > kCorrBatchMax) return cudaErrorInvalidValue;
  if (n_pix <= 0) return cudaSuccess;
  VisBatch b{};
  long long max_rows = 0;
  for (int i = 0; i < n_jobs; i++) {
    b.job[i] = jobs[i];
    max_rows = std::max(max_rows, jobs[i].n_rows);
  }
  if (max_rows <= 0) return cudaSuccess;
  const long long n_x = (max_rows + kVisBM - 1) / kVisBM;
  const int n_y = (n_pix + kVisBN - 1) / kVisBN;
  const long long n_tiles = n_x * n_y * n_jobs;
  if (n_tiles >= (1LL << 31)) return cudaErrorInvalidConfiguration;
  const int K = n_ant * (n_ant + 1);  // 2 n_pair real columns
  const long long grid = max_ctas > 0 && n_tiles > max_ctas ? max_ctas : n_tiles;
  k_beam_from_vis<<<(unsigned)grid, 256, 0, st>>>(b, K, wvis, beam_vis_ld(n_pix), n_pix, n_x, n_y,
                                                  n_jobs);
  return cudaGetLastError();
}

cudaError_t launch_beam_from_vis(const float2* V, const float* wvis, int n_ant, int n_pix,
                                 long long first, long long last, float* pow, cudaStream_t st,
                                 const int* dump_list, long long n_list) {
  if (n_pix <= 0 || (dump_list ? n_list <= 0 : last < first)) return cudaSuccess;
  const VisJob j{V, pow, first, dump_list ? n_list : last - first + 1, dump_list};
  return launch_beam_from_vis_batch(&j, 1, wvis, n_ant, n_pix, st);
}

// ------------------------------------------------------------------ beamform
// One CTA per (dump, 128 pixels).  Weights of the CTA's pixels live in shared
// memory antenna-major; a chunk of every antenna's voltages is staged and each
// thread forms its pixel's beam sample by sample.
constexpr int kBeamPix = 128;
constexpr int kBeamChunk = 128;

__global__ void __launch_bounds__(kBeamPix) k_beamform_simt(const float2* __restrict__ y,
                                                            long long n_samp, int M, int L,
                                                            long long m_base, long long first,
                                                            long long last,
                                                            const float2* __restrict__ W,
                                                            int n_pix, float* __restrict__ pow) {
  extern __shared__ float2 smem[];
  float2* sw = smem;                   // [M][kBeamPix]
  float2* sy = smem + M * kBeamPix;    // [M][kBeamChunk]
  const long long m = m_base + blockIdx.x;
  const int p = blockIdx.y * kBeamPix + threadIdx.x;
  float* out = pow + m * n_pix;
  if (m < first || m > last) {
    if (p < n_pix) out[p] = 0.f;
    return;
  }
  for (int a = 0; a < M; a++)
    sw[a * kBeamPix + threadIdx.x] = (p < n_pix) ? W[(long long)p * M + a] : make_float2(0.f, 0.f);
  float total = 0.f;
  const long long t0 = m * L;
  for (int c0 = 0; c0 < L; c0 += kBeamChunk) {
    const int len = (L - c0) < kBeamChunk ? (L - c0) : kBeamChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < M * len; i += blockDim.x) {
      int a = i / len, t = i % len;
      sy[a * kBeamChunk + t] = y[(long long)a * n_samp + t0 + c0 + t];
    }
    __syncthreads();
    float part = 0.f;
    for (int t = 0; t < len; t++) {
      float br = 0.f, bi = 0.f;
      for (int a = 0; a < M; a++) {
        float2 w = sw[a * kBeamPix + threadIdx.x];
        float2 v = sy[a * kBeamChunk + t];
        br = fmaf(w.x, v.x, fmaf(-w.y, v.y, br));
        bi = fmaf(w.x, v.y, fmaf(w.y, v.x, bi));
      }
      part = fmaf(br, br, fmaf(bi, bi, part));
    }
    total += part;
  }
  if (p < n_pix) out[p] = total;
}

cudaError_t launch_beamform_simt(const float2* y, long long n_samp, int n_ant, int dump_len,
                                 long long m_base, long long n_m, long long first, long long last,
                                 const float2* W, int n_pix, float* pow, cudaStream_t st) {
  size_t smem = (size_t)n_ant * (kBeamPix + kBeamChunk) * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_beamform_simt,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (n_m <= 0 || n_pix <= 0) return cudaSuccess;
  dim3 grid((unsigned)n_m, (n_pix + kBeamPix - 1) / kBeamPix);
  k_beamform_simt<<<grid, kBeamPix, smem, st>>>(y, n_samp, n_ant, dump_len, m_base, first, last,
                                                W, n_pix, pow);
  return cudaGetLastError();
}

}  // namespace chirp
