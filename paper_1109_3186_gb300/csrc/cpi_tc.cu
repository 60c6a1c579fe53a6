// cpi_tc.cu -- the Chirpolator pre-integrator's image (Eq. pth with the
// 2F+1-bin matched filter of Sec. 3.4, then E = |P|^2, Eq. eth) as a dense
// contraction on the tcgen05 tensor cores.
//
// Per trial DM d the image is  P[pix][m] = sum_{k, q} A[pix][k, q] X[m][k][q]
// over every bin k in [-K, K] and pair q, with the filter A zero except at
// the 2F+1 bins around each pair's tone (K0 .. K0 + 2F).  The sparse form
// gathers those bins per pixel on the CUDA cores; here A is densified once
// per plan (n_pix x (2K+1) n_pair complex per DM, about 3.4x the useful
// products on the bench workload) and the product runs as a GEMM in
// real-block form (row 2p gives Re P_p, row 2p+1 gives Im P_p; real K index
// 2 (k n_pair + q) + c for c = 0 real, 1 imaginary):
//   A[2p][2kk] = Re w, A[2p][2kk+1] = -Im w, A[2p+1][2kk] = Im w,
//   A[2p+1][2kk+1] = Re w,   B[2kk + c][m] = (Re, Im)_c X[m][kk].
// FP32 accuracy from BF16 operands: every operand is split into a BF16 head
// and tail, D = A_h B_h + A_h B_l + A_l B_h (the dropped A_l B_l is O(2^-16)),
// three MMAs per K step into one FP32 TMEM accumulator.
//
// Images (both K-major core matrices: 8 rows x 16 bytes, a row holds 8
// consecutive K values), laid out so that one bulk copy moves the head and
// tail of one (tile, K chunk):
//   A per DM: [row tile][K chunk][term][16 m-groups][4 k-groups][8 rows][8 bf16]
//   B per DM: [window tile][K chunk][term][32 n-groups][4 k-groups][8 windows][8 bf16]
// One CTA computes a 128-row x 256-window tile: a producer thread streams
// the K chunks (32 real K, 48 KB per stage, two stages), one thread issues
// the 6 MMAs of a chunk, four epilogue warps read the accumulator from TMEM,
// form |P|^2 of the pixel pairs of rows (lanes 2p, 2p+1) and write E.  Every
// wait is bounded; on a timeout the kernel raises *err, waits (bounded) for
// its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tc.cuh"

namespace chirp {

namespace {

constexpr int kCtM = 128;  // rows per tile (64 pixels, real and imaginary)
constexpr int kCtN = 256;  // windows per tile
constexpr int kCtK = 32;   // real K per stage: 2 MMA K steps of 16
constexpr int kCtStages = 2;
constexpr uint32_t kATerm = kCtM * kCtK * 2;  // 8 KB
constexpr uint32_t kBTerm = kCtN * kCtK * 2;  // 16 KB
constexpr uint32_t kAStage = 2 * kATerm;      // head + tail
constexpr uint32_t kBStage = 2 * kBTerm;
constexpr uint32_t kStage = kAStage + kBStage;  // 48 KB
constexpr int kCtThreads = 192;               // producer, MMA/TMEM, 4 epilogue warps
constexpr uint32_t kCtIdesc = tc::idesc_bf16_f32(kCtM, kCtN, false);  // A and B K-major

// byte offset of element (row, K) inside one term of a K chunk (K < 32)
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Dense A image of every DM from the sparse filter: W [n_dm][n_pair][nj][n_pix]
// complex, K0 [n_dm][n_pair][n_pix] first bin index in [0, nk).  One thread
// per (DM, pair, pixel); every (row, K) entry has exactly one writer, the
// rest of the image was cleared.
__global__ void k_cpi_tc_aimg(const float2* __restrict__ W, const short* __restrict__ K0,
                              int n_dm, int n_pair, int nj, int nk, int n_pix, int n_rt, int n_kc,
                              uint8_t* __restrict__ aimg) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_dm * n_pair * n_pix) return;
  const int pix = (int)(idx % n_pix);
  const long long dq = idx / n_pix;  // d n_pair + q
  const int q = (int)(dq % n_pair);
  const long long d = dq / n_pair;
  const int k0 = K0[dq * n_pix + pix];
  const size_t dm_bytes = (size_t)n_rt * n_kc * kAStage;
  uint8_t* base = aimg + (size_t)d * dm_bytes;
  const int row0 = 2 * pix;
  const int rt = row0 / kCtM, r0 = row0 % kCtM;  // rows r0, r0 + 1 of the same tile
  for (int j = 0; j < nj; j++) {
    const int k = k0 + j;
    if (k >= nk) break;
    const float2 w = W[(dq * nj + j) * n_pix + pix];
    const long long kk = (long long)k * n_pair + q;
    const int K = (int)(2 * kk);  // real index of Re; Re+1 = Im (same chunk: K is even)
    const int kc = K / kCtK, kin = K % kCtK;
    uint8_t* chunk = base + ((size_t)rt * n_kc + kc) * kAStage;
    const float vals[2][2] = {{w.x, -w.y}, {w.y, w.x}};  // [row offset][K offset]
#pragma unroll
    for (int dr = 0; dr < 2; dr++)
#pragma unroll
      for (int dk = 0; dk < 2; dk++) {
        __nv_bfloat16 h, l;
        split_bf16(vals[dr][dk], h, l);
        const uint32_t off = core_off(r0 + dr, kin + dk);
        *reinterpret_cast<__nv_bfloat16*>(chunk + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(chunk + kATerm + off) = l;
      }
  }
}

// B image of every DM from the window DFTs X [n_dm][n_blk][nk n_pair] complex:
// one thread per (DM, window, 4 consecutive kk) writes one 16-byte row of the
// head and one of the tail (8 real K: 4 complex values).  K beyond the last
// pair's last bin (padding of the final chunk) stays zero.
__global__ void k_cpi_tc_bimg(const float2* __restrict__ X, int n_dm, long long n_blk, int n_kk,
                              int n_nt, int n_kc, uint8_t* __restrict__ bimg) {
  const int groups = n_kc * (kCtK / 8);  // 16-byte rows per window
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_dm * n_blk * groups) return;
  const int g = (int)(idx % groups);
  const long long dm_ = idx / groups;  // d n_blk + m
  const long long m = dm_ % n_blk, d = dm_ / n_blk;
  const int kc = g / (kCtK / 8), kg = g % (kCtK / 8);
  const int nt = (int)(m / kCtN), mr = (int)(m % kCtN);
  __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int kk = 4 * g + i;
    const float2 v = kk < n_kk ? X[dm_ * n_kk + kk] : make_float2(0.f, 0.f);
    split_bf16(v.x, h[2 * i], l[2 * i]);
    split_bf16(v.y, h[2 * i + 1], l[2 * i + 1]);
  }
  const size_t dm_bytes = (size_t)n_nt * n_kc * kBStage;
  uint8_t* chunk = bimg + (size_t)d * dm_bytes + ((size_t)nt * n_kc + kc) * kBStage;
  const uint32_t off = (uint32_t)((((mr >> 3) * 4 + kg) * 128) + (mr & 7) * 16);
  *reinterpret_cast<uint4*>(chunk + off) = *reinterpret_cast<const uint4*>(h);
  *reinterpret_cast<uint4*>(chunk + kBTerm + off) = *reinterpret_cast<const uint4*>(l);
}

struct CpiTcArgs {
  const uint8_t* aimg;
  const uint8_t* bimg;
  const int* n_win;
  float* E;
  int* err;
  long long n_blk;
  int n_pix, n_rt, n_nt, n_kc;
};

// grid (window tile, row tile, DM): the window tiles of a row tile run
// together and share its A chunks in L2.
__global__ void __launch_bounds__(kCtThreads) k_cpi_tc(CpiTcArgs args) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kCtStages * kStage);
  uint64_t* full = bars;                  // [kCtStages]
  uint64_t* empty = bars + kCtStages;     // [kCtStages]
  uint64_t* accf = bars + 2 * kCtStages;  // accumulator ready
  uint64_t* drain = accf + 1;             // MMA queue drained (teardown)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nt = blockIdx.x, rt = blockIdx.y;
  const long long d = blockIdx.z;
  const long long m0 = (long long)nt * kCtN;
  const int nw = args.n_win[d];
  const long long m_end = m0 + kCtN < args.n_blk ? m0 + kCtN : args.n_blk;
  const bool work = m_end - 1 >= nw - 1;  // some window of the tile is complete
  const int n_kc = args.n_kc;
  const uint8_t* a_src = args.aimg + ((size_t)d * args.n_rt + rt) * (size_t)n_kc * kAStage;
  const uint8_t* b_src = args.bimg + ((size_t)d * args.n_nt + nt) * (size_t)n_kc * kBStage;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kCtStages; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(accf, 1);
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 256);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  auto raise = [&]() {
    *abort_flag = 1;
    atomicExch(args.err, 1);
  };

  if (work) {
    if (warp == 0 && lane == 0) {
      // ------------------------------------------------------ producer
      long long issued = 0;
      for (int kc = 0; kc < n_kc; kc++) {
        const int s = kc % kCtStages;
        const uint32_t ph = (uint32_t)((kc / kCtStages) & 1);
        if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
          raise();
          break;
        }
        uint8_t* st = smem + (size_t)s * kStage;
        tc::mbar_arrive_expect_tx(&full[s], kStage);
        tc::bulk_g2s(st, a_src + (size_t)kc * kAStage, kAStage, &full[s]);
        tc::bulk_g2s(st + kAStage, b_src + (size_t)kc * kBStage, kBStage, &full[s]);
        issued = kc + 1;
      }
      if (*abort_flag) {  // let every copy this thread issued land before the CTA goes away
        for (long long i = issued > kCtStages ? issued - kCtStages : 0; i < issued; i++)
          tc::mbar_wait(&full[i % kCtStages], (uint32_t)((i / kCtStages) & 1), nullptr, 1u << 22);
      }
    } else if (warp == 1 && lane == 0) {
      // ------------------------------------------------------ MMA issuer
      bool ok = true;
      for (int kc = 0; kc < n_kc && ok; kc++) {
        const int s = kc % kCtStages;
        const uint32_t ph = (uint32_t)((kc / kCtStages) & 1);
        if (!tc::mbar_wait(&full[s], ph, abort_flag)) {
          raise();
          ok = false;
          break;
        }
        tc::fence_after();
        const uint32_t sa = tc::smem_u32(smem + (size_t)s * kStage);
        const uint32_t sb = sa + kAStage;
#pragma unroll
        for (int ks = 0; ks < kCtK / 16; ks++) {
          // K step ks: 2 core-matrix columns (256 bytes) into the chunk
          const uint64_t ah = tc::sdesc(sa + ks * 256, 128u, 512u);
          const uint64_t al = tc::sdesc(sa + kATerm + ks * 256, 128u, 512u);
          const uint64_t bh = tc::sdesc(sb + ks * 256, 128u, 512u);
          const uint64_t bl = tc::sdesc(sb + kBTerm + ks * 256, 128u, 512u);
          const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
          tc::mma_bf16(tmem, ah, bh, kCtIdesc, acc0);
          tc::mma_bf16(tmem, ah, bl, kCtIdesc, 1u);
          tc::mma_bf16(tmem, al, bh, kCtIdesc, 1u);
        }
        tc::mma_commit(&empty[s]);
      }
      if (ok) tc::mma_commit(accf);
      // nothing may be in flight when TMEM is released
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0, nullptr, 1u << 22);
    } else if (warp >= 2) {
      // ------------------------------------------------------ epilogue
      const int q = warp & 3;  // TMEM lane quarter of this warp
      const int row = 32 * q + lane;
      const bool ok = tc::mbar_wait(accf, 0, abort_flag, 1u << 26);
      if (!ok) raise();
      tc::fence_after();
      const int pix = (rt * kCtM + row) >> 1;
      for (int c = 0; c < kCtN / 32; c++) {
        float v[32];
        if (ok) tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * c), v);
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const float e = v[j] * v[j];
          v[j] = e + __shfl_xor_sync(0xffffffffu, e, 1);
        }
        if (ok && !(lane & 1) && pix < args.n_pix) {
#pragma unroll
          for (int j = 0; j < 32; j++) {
            const long long m = m0 + 32 * c + j;
            if (m < m_end)
              args.E[(d * args.n_blk + m) * args.n_pix + pix] = m >= nw - 1 ? v[j] : 0.f;
          }
        }
      }
    }
  } else if (warp >= 2) {
    // every window of the tile is incomplete: zeros
    const int row = 32 * (warp & 3) + lane;
    const int pix = (rt * kCtM + row) >> 1;
    if (!(lane & 1) && pix < args.n_pix)
      for (long long m = m0; m < m_end; m++) args.E[(d * args.n_blk + m) * args.n_pix + pix] = 0.f;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

long long cpi_tc_a_bytes(int n_dm, int n_pix, int nk, int n_pair) {
  const long long n_rt = (2LL * n_pix + kCtM - 1) / kCtM;
  const long long n_kc = (2LL * nk * n_pair + kCtK - 1) / kCtK;
  return (long long)n_dm * n_rt * n_kc * kAStage;
}

long long cpi_tc_b_bytes(int n_dm, long long n_blk, int nk, int n_pair) {
  const long long n_nt = (n_blk + kCtN - 1) / kCtN;
  const long long n_kc = (2LL * nk * n_pair + kCtK - 1) / kCtK;
  return (long long)n_dm * n_nt * n_kc * kBStage;
}

cudaError_t launch_cpi_tc_aimg(const float2* W, const short* K0, int n_dm, int n_pair, int nj,
                               int nk, int n_pix, uint8_t* aimg, cudaStream_t st) {
  const int n_rt = (2 * n_pix + kCtM - 1) / kCtM;
  const int n_kc = (2 * nk * n_pair + kCtK - 1) / kCtK;
  cudaError_t e = cudaMemsetAsync(aimg, 0, (size_t)cpi_tc_a_bytes(n_dm, n_pix, nk, n_pair), st);
  if (e != cudaSuccess) return e;
  const long long n = (long long)n_dm * n_pair * n_pix;
  k_cpi_tc_aimg<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, K0, n_dm, n_pair, nj, nk, n_pix,
                                                            n_rt, n_kc, aimg);
  return cudaGetLastError();
}

cudaError_t launch_cpi_tc_image(const float2* X, uint8_t* bimg, const uint8_t* aimg,
                                const int* n_win, int n_dm, long long n_blk, int nk, int n_pair,
                                int n_pix, float* E, int* err, cudaStream_t st) {
  const int n_kk = nk * n_pair;
  const int n_kc = (2 * n_kk + kCtK - 1) / kCtK;
  const int n_nt = (int)((n_blk + kCtN - 1) / kCtN);
  const int n_rt = (2 * n_pix + kCtM - 1) / kCtM;
  if (n_nt > 65535 || n_rt > 65535 || n_dm > 65535) return cudaErrorInvalidConfiguration;
  // windows of the last tile beyond n_blk read as zeros
  if (n_blk % kCtN) {
    cudaError_t e = cudaMemsetAsync(bimg, 0, (size_t)cpi_tc_b_bytes(n_dm, n_blk, nk, n_pair), st);
    if (e != cudaSuccess) return e;
  }
  const long long nb = (long long)n_dm * n_blk * n_kc * (kCtK / 8);
  k_cpi_tc_bimg<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(X, n_dm, n_blk, n_kk, n_nt, n_kc,
                                                             bimg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)kCtStages * kStage + 64;
  e = cudaFuncSetAttribute(k_cpi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  CpiTcArgs a{aimg, bimg, n_win, E, err, n_blk, n_pix, n_rt, n_nt, n_kc};
  k_cpi_tc<<<dim3((unsigned)n_nt, (unsigned)n_rt, (unsigned)n_dm), kCtThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chirp
