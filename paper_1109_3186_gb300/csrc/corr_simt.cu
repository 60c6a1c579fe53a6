// corr_simt.cu -- Chirpolator back-end on the CUDA cores with staged input.
//
// Per dump m the zero-lag products V_pq = sum_{t in dump} y_p(t) y_q(t)^*
// (p <= q, autos included; the pair mixing of Eq. xpq integrated and
// dumped), in FP32, for up to kScMaxAnt antennas.  The plain kernel of
// backends.cu loads y with ordinary loads one dump per CTA and is bound by
// memory latency; here a loader warp streams the dumps' antenna rows into a
// ring of shared-memory stages with bulk copies, several chunks ahead, and
// the compute warps read them from shared memory:
//  - the M x M product is cut into 4 x 4 antenna tiles on or above the
//    diagonal; each tile pair has K = floor(12 / tiles) compute warps, warp
//    k of a tile pair taking the samples lane + 32 (k + K j) of every chunk
//    and keeping the tile's 16 complex products in registers over the dump;
//  - a dump is read in chunks of up to kc samples from its start (any even
//    dump length); after its last chunk every warp sums its lanes with
//    shuffles, the K partials of a tile pair are added in a fixed order
//    through shared memory and written out.
// Every wait is bounded; a wait that gives up raises the plan's error word
// and the CTA winds down (all compute warps take the same stop decision at
// each dump end, and the loader waits for its copies in flight before the
// CTA leaves).
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tc.cuh"

namespace chirp {

namespace {

constexpr int kScTile = 4;
constexpr int kScMaxAnt = 16;                    // at most 10 tile pairs for 12 warps
constexpr int kScCompWarps = 12;
constexpr int kScLoaderWarp = kScCompWarps;
constexpr int kScThreads = 32 * (kScCompWarps + 1);
constexpr int kScStages = 4;
constexpr uint32_t kScStageBudget = 40u * 1024u;  // bytes of one raw stage at most

struct ScArgs {
  const float2* y;
  long long n_samp;
  float2* vis;        // this DM: [n_dump][n_pair]
  int* err;
  long long first;    // first dump of the range (all dumps of the range are valid)
  const int* dump_list;  // or NULL; else the n_dumps (valid) dumps to correlate
  long long n_dumps;
  long long dumps_per_cta;
  int M, L, kc, n_tp, K;
  uint32_t stage_bytes, part_off, bar_off;
};

__global__ void __launch_bounds__(kScThreads, 1) k_correlate_staged(ScArgs args) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* stages = smem;
  float2* part = (float2*)(smem + args.part_off);   // [compute warp][16]
  uint64_t* full = (uint64_t*)(smem + args.bar_off);  // [kScStages]
  uint64_t* empty = full + kScStages;                 // [kScStages]
  volatile int* abort_flag = (volatile int*)(empty + kScStages);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int M = args.M, L = args.L, kc = args.kc;
  // positions [j_a, j_b) of the range or list; dump of position j
  const long long j_a = (long long)blockIdx.x * args.dumps_per_cta;
  const long long j_b = min(j_a + args.dumps_per_cta, args.n_dumps);
  auto dump_of = [&](long long j) -> long long {
    return args.dump_list ? (long long)args.dump_list[j] : args.first + j;
  };
  const int chunks_per_dump = (L + kc - 1) / kc;
  const long long n_chunks = j_b > j_a ? (j_b - j_a) * chunks_per_dump : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kScStages; s++) {
      tc::mbar_init(&full[s], 1);              // the loader's expect-tx arrival
      tc::mbar_init(&empty[s], kScCompWarps);  // one arrival per compute warp
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  auto raise = [&]() {
    *abort_flag = 1;
    atomicExch(args.err, 1);
  };

  if (warp == kScLoaderWarp) {
    // ------------------------------------------------------ loader
    if (lane == 0) {
      long long issued = 0;
      for (long long i = 0; i < n_chunks; i++) {
        const int s = (int)(i % kScStages);
        const uint32_t ph = (uint32_t)((i / kScStages) & 1);
        if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
          raise();
          break;
        }
        const long long m = dump_of(j_a + i / chunks_per_dump);
        const int c = (int)(i % chunks_per_dump);
        const int n = min(kc, L - c * kc);  // even: 16-byte rows
        const uint32_t bytes = (uint32_t)n * 8u;
        tc::mbar_arrive_expect_tx(&full[s], bytes * (uint32_t)M);
        for (int a = 0; a < M; a++)
          tc::bulk_g2s(stages + (size_t)s * args.stage_bytes + (size_t)a * kc * 8,
                       args.y + (long long)a * args.n_samp + m * L + (long long)c * kc, bytes,
                       &full[s]);
        issued = i + 1;
      }
      for (long long k = issued > kScStages ? issued - kScStages : 0; k < issued; k++)
        tc::mbar_wait(&full[(int)(k % kScStages)], (uint32_t)((k / kScStages) & 1), nullptr,
                      1u << 22);
    }
  } else {
    // ------------------------------------------------------ compute warps
    const int tp = warp / args.K, k = warp % args.K;
    const bool active = tp < args.n_tp;
    const int nt = (M + kScTile - 1) / kScTile;
    int ti = 0, tj = 0;
    if (active) {
      int rem = tp;
      while (rem >= nt - ti) {
        rem -= nt - ti;
        ti++;
      }
      tj = ti + rem;
    }
    int ri[kScTile], rj[kScTile];  // stage rows (element offsets) of the tile's antennas
    bool vi[kScTile], vj[kScTile];
#pragma unroll
    for (int a = 0; a < kScTile; a++) {
      const int ai = ti * kScTile + a, aj = tj * kScTile + a;
      vi[a] = ai < M;
      vj[a] = aj < M;
      ri[a] = (vi[a] ? ai : 0) * kc;
      rj[a] = (vj[a] ? aj : 0) * kc;
    }
    const int n_pair = M * (M + 1) / 2;
    bool aborted = false;
    long long i = 0;
    for (long long j = j_a; j < j_b; j++) {
      const long long m = dump_of(j);
      float2 acc[kScTile][kScTile];
#pragma unroll
      for (int a = 0; a < kScTile; a++)
#pragma unroll
        for (int b = 0; b < kScTile; b++) acc[a][b] = make_float2(0.f, 0.f);
      for (int c = 0; c < chunks_per_dump; c++, i++) {
        const int s = (int)(i % kScStages);
        const uint32_t ph = (uint32_t)((i / kScStages) & 1);
        if (!aborted && !tc::mbar_wait(&full[s], ph, abort_flag)) {
          raise();
          aborted = true;
        }
        if (!aborted && active) {
          const int n = min(kc, L - c * kc);
          const float2* st = (const float2*)(stages + (size_t)s * args.stage_bytes);
#pragma unroll 2
          for (int t = lane + 32 * k; t < n; t += 32 * args.K) {
            float2 u[kScTile], w[kScTile];
#pragma unroll
            for (int a = 0; a < kScTile; a++) {
              u[a] = vi[a] ? st[ri[a] + t] : make_float2(0.f, 0.f);
              w[a] = vj[a] ? st[rj[a] + t] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int a = 0; a < kScTile; a++)
#pragma unroll
              for (int b = 0; b < kScTile; b++) {  // u_a * conj(w_b)
                acc[a][b].x = fmaf(u[a].x, w[b].x, fmaf(u[a].y, w[b].y, acc[a][b].x));
                acc[a][b].y = fmaf(u[a].y, w[b].x, fmaf(-u[a].x, w[b].y, acc[a][b].y));
              }
          }
        }
        __syncwarp();
        if (!aborted && lane == 0) tc::mbar_arrive(&empty[s]);
      }
      // the warp's lane partials -> one sum per product, kept by every lane
#pragma unroll
      for (int a = 0; a < kScTile; a++)
#pragma unroll
        for (int b = 0; b < kScTile; b++)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            acc[a][b].x += __shfl_xor_sync(0xffffffffu, acc[a][b].x, o);
            acc[a][b].y += __shfl_xor_sync(0xffffffffu, acc[a][b].y, o);
          }
      if (lane == 0)
#pragma unroll
        for (int a = 0; a < kScTile; a++)
#pragma unroll
          for (int b = 0; b < kScTile; b++) part[warp * 16 + a * kScTile + b] = acc[a][b];
      // every compute warp takes the same stop decision (an OR of their views)
      uint32_t stop_u;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\t"
          "setp.ne.u32 p, %1, 0;\n\t"
          "bar.red.or.pred q, 1, %2, p;\n\t"
          "selp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(stop_u)
          : "r"((uint32_t)(aborted || *abort_flag != 0)), "r"(32 * kScCompWarps)
          : "memory");
      const bool stop = stop_u != 0;
      if (!stop && active && k == 0 && lane < 16) {
        // the K warps of this tile pair, added in order
        float2 v = part[warp * 16 + lane];
        for (int kk = 1; kk < args.K; kk++) {
          const float2 o = part[(warp + kk) * 16 + lane];
          v.x += o.x;
          v.y += o.y;
        }
        const int p = ti * kScTile + lane / kScTile, q = tj * kScTile + lane % kScTile;
        if (p < M && q < M && p <= q) args.vis[m * n_pair + p * M - p * (p - 1) / 2 + (q - p)] = v;
      }
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kScCompWarps) : "memory");  // part is reused
      if (stop) break;
    }
  }
}

}  // namespace

bool correlate_staged_supported(int n_ant, int dump_len, long long n_samp, const void* y) {
  return n_ant >= 1 && n_ant <= kScMaxAnt && dump_len >= 2 && dump_len % 2 == 0 &&
         n_samp % 2 == 0 && ((uintptr_t)y % 16) == 0;
}

cudaError_t launch_correlate_staged(const float2* y, long long n_samp, int n_ant, int dump_len,
                                    long long first, long long n_dumps, float2* vis, int* err,
                                    cudaStream_t st, const int* dump_list) {
  if (n_dumps <= 0) return cudaSuccess;
  if (!correlate_staged_supported(n_ant, dump_len, n_samp, y) || err == nullptr)
    return cudaErrorInvalidValue;
  ScArgs a;
  a.y = y;
  a.n_samp = n_samp;
  a.vis = vis;
  a.err = err;
  a.first = first;
  a.dump_list = dump_list;
  a.n_dumps = n_dumps;
  a.M = n_ant;
  a.L = dump_len;
  int kc = (int)(kScStageBudget / ((uint32_t)n_ant * 8u)) / 32 * 32;
  if (kc > 256) kc = 256;
  a.kc = kc;
  const int nt = (n_ant + kScTile - 1) / kScTile;
  a.n_tp = nt * (nt + 1) / 2;
  a.K = kScCompWarps / a.n_tp;
  a.stage_bytes = ((uint32_t)n_ant * (uint32_t)kc * 8u + 127u) & ~127u;
  a.part_off = kScStages * a.stage_bytes;
  a.bar_off = a.part_off + kScCompWarps * 16 * (uint32_t)sizeof(float2);
  const uint32_t smem = a.bar_off + 2 * kScStages * 8 + 16;
  cudaError_t e = cudaFuncSetAttribute(k_correlate_staged,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // as many CTAs as are resident at once (registers, shared memory,
  // threads), the dumps split evenly among them
  int dev = 0, n_sm = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_correlate_staged, kScThreads,
                                                      smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long grid = (long long)n_sm * per_sm;
  if (grid > n_dumps) grid = n_dumps;
  a.dumps_per_cta = (n_dumps + grid - 1) / grid;
  grid = (n_dumps + a.dumps_per_cta - 1) / a.dumps_per_cta;
  k_correlate_staged<<<(unsigned)grid, kScThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chirp
