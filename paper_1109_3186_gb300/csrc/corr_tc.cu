// corr_tc.cu -- Chirpolator back-end on the tcgen05 tensor cores.
//
// Per dump m of a DM the zero-lag cross products of every antenna pair,
//   V_pq = sum_{t in dump} y_p(t) y_q(t)^*   (p <= q, autos included),
// i.e. the pair mixing of Eq. xpq integrated and dumped: a Hermitian rank-L
// update of the M antenna voltages.  Real form: with the 2M real rows
// r_k (k = 2a + c: c = 0 real, 1 imaginary part of antenna a) and their Gram
// matrix Gm(k, l) = sum_t r_k(t) r_l(t),
//   Re V_ab = Gm(2a, 2b) + Gm(2a+1, 2b+1),   Im V_ab = Gm(2a+1, 2b) - Gm(2a, 2b+1).
// FP32 accuracy from BF16 tensor cores: r = h + l (BF16 head and tail), and
//   Gm ~ H H^T + L H^T + (L H^T)^T     (L L^T is O(2^-16) and dropped),
// so ONE contraction D = [H; L] H^T (rows: the head, then the tail rows;
// columns: the head rows; K: the dump's samples) holds all three products.
// One term (reduced precision): D = H H^T.
//
// Rows are grouped 8 per 4 antennas (G = ceil(M / 4) groups): head rows
// 0 .. 8G-1 (rows of absent antennas zero), tail rows 8G .. 16G-1.
//
// The kernel reads the FP32 voltages y [M][N] once: a loader warp streams
// each chunk's antenna rows into a ring of raw FP32 stages with bulk copies
// (several chunks ahead, so that enough bytes are in flight to stream HBM);
// where the rows are not 16-byte aligned (odd N) or the ring does not fit,
// the producers load y themselves.  Two groups of 4
// producer warps convert alternate chunks of kc samples into the BF16
// operand (K-major, no swizzle: core matrices of 8 rows x 8 samples; the
// k-groups of a row group 144 B apart, row groups SBO apart) in a ring of
// shared-memory stages.  One thread issues the MMAs: per 16-sample K step
// and 128-row tile one tcgen05.mma (N = head rows rounded up to 16) into a
// TMEM accumulator.  The tensor core's FP32 accumulation over hundreds of K
// steps drifts by ~1e-5 relative (measured), so a dump is summed in segments
// of one chunk (at most 256 samples): each segment has its own accumulator,
// and four epilogue warps add finished segments into FP32 running sums in
// shared memory and, at the end of the dump, form the M(M+1)/2
// visibilities.  Chunk and dump boundaries line up: dump_len is a multiple
// of the chunk length, or divides it.  The MMA reads 128 rows per row tile; rows past
// the used ones read whatever lies after the stage (finite or not) and only
// produce accumulator rows that are never read.  Every wait is bounded; on a
// timeout the kernel raises *err and winds down.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tc.cuh"

namespace chirp {

namespace {

constexpr int kProdWarps = 8;                 // two groups of 4
constexpr int kIssuerWarp = kProdWarps;       // also allocates TMEM
constexpr int kEpiWarp0 = kProdWarps + 1;     // 4 epilogue warps
constexpr int kLoaderWarp = kEpiWarp0 + 4;    // bulk copies of the raw voltages
constexpr int kCorrThreads = 32 * (kLoaderWarp + 1);
constexpr int kMaxStages = 4;
constexpr int kMaxAcc = 4;
constexpr int kMaxRaw = 4;
constexpr uint32_t kCorrSmemLimit = 227u * 1024u;
// Stride between the K-adjacent core matrices of a row group: 128 B plus a
// 16-byte gap, so that the producer lanes writing consecutive 8-sample
// groups of one row hit different banks.
constexpr uint32_t kLbo = 144;
constexpr int kBatch = 4;                     // producer items loaded together

struct CorrGeom {
  int G, KR, n_rt, NC, Npad, nacc, kc, nst, nraw;
  uint32_t sbo, stage_stride, stage_region, dsm_off, bar_off, total, raw_off, raw_stride;
};

// Stage plan for chunks of kc samples and nst stages; nraw raw FP32 stages
// (M rows of kc float2 each) after the barriers, or none.  Returns the bytes.
__host__ __device__ inline uint32_t corr_plan(CorrGeom* g, int M, int kc, int nst, int nraw) {
  g->kc = kc;
  g->nst = nst;
  g->sbo = (uint32_t)(kc / 8) * kLbo;
  const uint32_t groups = (uint32_t)(g->KR + 7) / 8;
  g->stage_stride = groups * g->sbo;
  // the MMA windows of the last stage may run into the staging, the
  // barriers and the raw ring (only accumulator rows that are never read
  // come from there): they only have to stay inside the allocation
  const uint32_t window = (uint32_t)g->n_rt * 16u * g->sbo;
  g->stage_region = (uint32_t)nst * g->stage_stride;
  g->dsm_off = g->stage_region;
  g->bar_off = (g->dsm_off + (uint32_t)g->KR * (g->NC + 1) * 4u + 15u) & ~15u;
  g->nraw = nraw;
  g->raw_stride = ((uint32_t)M * (uint32_t)kc * 8u + 127u) & ~127u;
  g->raw_off = (g->bar_off + 256u + 127u) & ~127u;
  const uint32_t end = nraw > 0 ? g->raw_off + (uint32_t)nraw * g->raw_stride : g->bar_off + 256;
  const uint32_t last_window_end = (uint32_t)(nst - 1) * g->stage_stride + window;
  g->total = end > last_window_end ? end : last_window_end;
  return g->total;
}

// Shared-memory plan: the stages (each KR rows of kc samples), the staging
// of one accumulator (KR x (NC + 1) floats) and the barriers, with the
// allocation long enough for the 128-row windows the MMAs read; then, with
// the same chunk length, as deep a raw ring as fits (giving up stages down
// to two for it), else none.
__host__ __device__ inline bool corr_geom(int M, int terms, int L, CorrGeom* g) {
  if (L % 16 != 0) return false;
  g->G = (M + 3) / 4;
  g->NC = 8 * g->G;
  g->KR = terms == 3 ? 16 * g->G : 8 * g->G;
  g->n_rt = (g->KR + 127) / 128;
  g->Npad = (g->NC + 15) / 16 * 16;
  if (g->Npad > 256) return false;
  g->nacc = 512 / (g->n_rt * g->Npad);
  if (g->nacc > kMaxAcc) g->nacc = kMaxAcc;
  if (g->nacc < 1) return false;
  for (int kc = 256; kc >= 128; kc -= 128) {
    if (L % kc != 0 && kc % L != 0) continue;  // chunks and dumps must line up
    for (int nst = kMaxStages; nst >= 2; nst--) {
      if (corr_plan(g, M, kc, nst, 0) > kCorrSmemLimit) continue;
      for (int ns = nst; ns >= 2; ns--)
        for (int nraw = kMaxRaw; nraw >= 2; nraw--)
          if (corr_plan(g, M, kc, ns, nraw) <= kCorrSmemLimit) return true;
      corr_plan(g, M, kc, nst, 0);
      return true;
    }
  }
  return false;
}

struct CorrArgs {
  const float2* y;
  long long n_samp;
  float2* vis;          // this DM: [n_dump][n_pair]
  int* err;
  long long first;      // first dump of the range
  long long n_dumps;
  long long dumps_per_cta;
  int M, L, terms;
  int raw_path;         // the loader streams y into the raw ring (rows 16-byte aligned)
  CorrGeom g;
};

__global__ void __launch_bounds__(kCorrThreads, 1) k_corr_tc(CorrArgs args) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const CorrGeom& g = args.g;
  uint8_t* stages = smem;
  float* dsm = (float*)(smem + g.dsm_off);
  uint64_t* full = (uint64_t*)(smem + g.bar_off);  // [kMaxStages]
  uint64_t* empty = full + kMaxStages;              // [kMaxStages]
  uint64_t* accf = empty + kMaxStages;              // [kMaxAcc]
  uint64_t* acce = accf + kMaxAcc;                  // [kMaxAcc]
  uint64_t* drain = acce + kMaxAcc;
  uint64_t* raw_full = drain + 1;                   // [kMaxRaw]
  uint64_t* raw_empty = raw_full + kMaxRaw;         // [kMaxRaw]
  uint32_t* tmem_slot = (uint32_t*)(raw_empty + kMaxRaw);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int M = args.M, L = args.L, nst = g.nst, kc = g.kc;
  const long long m_a = args.first + (long long)blockIdx.x * args.dumps_per_cta;
  const long long m_b = min(m_a + args.dumps_per_cta, args.first + args.n_dumps);
  const long long ta = m_a * L, tb = m_b * L;
  const long long n_chunks = m_b > m_a ? (tb - ta + kc - 1) / kc : 0;

  // zero the stage region once: rows of absent antennas, and rows past the
  // used ones inside the MMA windows, must hold finite values
  for (uint32_t i = threadIdx.x; i < g.stage_region / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(stages)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; s++) {
      tc::mbar_init(&full[s], 4 * 32);  // the threads of one producer group
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < g.nacc; a++) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], 4);  // every epilogue warp arrives once
    }
    tc::mbar_init(drain, 1);
    for (int r = 0; r < kMaxRaw; r++) {
      tc::mbar_init(&raw_full[r], 1);      // the loader's expect-tx arrival
      tc::mbar_init(&raw_empty[r], 4 * 32);  // the threads of one producer group
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == kIssuerWarp) tc::tmem_alloc(tmem_slot, 512);
  tc::fence_proxy_async_smem();  // the zeroed stages are read by the tensor core
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  auto raise = [&]() {
    *abort_flag = 1;
    atomicExch(args.err, 1);
  };

  if (n_chunks > 0) {
    if (warp < kProdWarps) {
      // ------------------------------------------------------ producers
      // group pg fills chunks i = pg, pg + 2, ...; item (antenna a, 8-sample
      // group e) -> 4 rows (head re/im, tail re/im) of 16 bytes each
      const int pg = warp / 4, ptid = threadIdx.x % 128;
      const int groups_per_chunk = kc / 8;
      const uint8_t* raw = smem + g.raw_off;
      for (long long i = pg; i < n_chunks; i += 2) {
        const int s = (int)(i % nst);
        const uint32_t ph = (uint32_t)((i / nst) & 1);
        if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
          raise();
          break;
        }
        const long long tc0 = ta + i * kc;
        const int n_groups = (int)min((long long)groups_per_chunk, (tb - tc0) / 8);
        uint8_t* st = stages + (size_t)s * g.stage_stride;
        const int n_items = M * n_groups;
        // samples 8e .. 8e + 7 of antenna a (as 4 float4: re, im of two
        // samples each) -> the 4 rows of the item
        auto convert = [&](int a, int e, const float4 (&v4)[4]) {
          uint32_t hr[4], hi[4], lr[4], li[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {  // samples 2j, 2j + 1 of the group
            const float4 v = v4[j];
            const __nv_bfloat162 h_r = __floats2bfloat162_rn(v.x, v.z);
            const __nv_bfloat162 h_i = __floats2bfloat162_rn(v.y, v.w);
            const float2 fr = __bfloat1622float2(h_r), fi = __bfloat1622float2(h_i);
            const __nv_bfloat162 l_r = __floats2bfloat162_rn(v.x - fr.x, v.z - fr.y);
            const __nv_bfloat162 l_i = __floats2bfloat162_rn(v.y - fi.x, v.w - fi.y);
            hr[j] = *reinterpret_cast<const uint32_t*>(&h_r);
            hi[j] = *reinterpret_cast<const uint32_t*>(&h_i);
            lr[j] = *reinterpret_cast<const uint32_t*>(&l_r);
            li[j] = *reinterpret_cast<const uint32_t*>(&l_i);
          }
          auto put = [&](int row, const uint32_t (&w)[4]) {
            *reinterpret_cast<uint4*>(st + (size_t)(row / 8) * g.sbo + (size_t)e * kLbo +
                                      (size_t)(row % 8) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
          };
          put(2 * a, hr);
          put(2 * a + 1, hi);
          if (args.terms == 3) {
            put(g.NC + 2 * a, lr);
            put(g.NC + 2 * a + 1, li);
          }
        };
        if (args.raw_path) {
          // the chunk's rows arrive in raw stage r by bulk copy (a ring in
          // chunk order; each phase of a slot has one consumer group)
          const int r = (int)(i % g.nraw);
          const uint32_t rph = (uint32_t)((i / g.nraw) & 1);
          if (!tc::mbar_wait(&raw_full[r], rph, abort_flag)) {
            raise();
            break;
          }
          const uint8_t* rs = raw + (size_t)r * g.raw_stride;
          for (int it = ptid; it < n_items; it += 128) {
            const int a = it / n_groups, e = it % n_groups;
            const float4* src = reinterpret_cast<const float4*>(rs + ((size_t)a * kc + 8 * e) * 8);
            float4 v4[4];
#pragma unroll
            for (int j = 0; j < 4; j++) v4[j] = src[j];
            convert(a, e, v4);
          }
          tc::mbar_arrive(&raw_empty[r]);
        } else {
          // items are handled in batches of kBatch per thread whose loads are all
          // issued before any is used (16-byte loads where the row is aligned),
          // so that more bytes are in flight
          for (int it0 = 0; it0 < n_items; it0 += 128 * kBatch) {
            float4 rawv[kBatch][4];
#pragma unroll
            for (int b = 0; b < kBatch; b++) {
              const int it = it0 + b * 128 + ptid;
              if (it < n_items) {
                const int a = it / n_groups, e = it % n_groups;
                const long long off = (long long)a * args.n_samp + tc0 + 8 * e;
                if ((off & 1) == 0) {
                  const float4* src = reinterpret_cast<const float4*>(args.y + off);
#pragma unroll
                  for (int j = 0; j < 4; j++) rawv[b][j] = src[j];
                } else {
                  const float2* src = args.y + off;
#pragma unroll
                  for (int j = 0; j < 4; j++) {
                    const float2 u = src[2 * j], w = src[2 * j + 1];
                    rawv[b][j] = make_float4(u.x, u.y, w.x, w.y);
                  }
                }
              }
            }
#pragma unroll
            for (int b = 0; b < kBatch; b++) {
              const int it = it0 + b * 128 + ptid;
              if (it >= n_items) continue;
              convert(it / n_groups, it % n_groups, rawv[b]);
            }
          }
        }
        tc::fence_proxy_async_smem();  // generic-proxy writes -> tensor-core reads
        tc::mbar_arrive(&full[s]);
      }
    } else if (warp == kIssuerWarp && lane == 0) {
      // ------------------------------------------------------ MMA issuer
      // Chunks and accumulation segments line up (dump_len a multiple of the
      // chunk length, or the chunk a multiple of dump_len): a segment is
      // seg_ks = min(kc, L) / 16 K steps, issued back to back from
      // descriptors advanced by constant offsets.
      const uint32_t idesc = tc::idesc_bf16_f32(128, g.Npad);
      const uint64_t desc0 = tc::sdesc(tc::smem_u32(stages), kLbo, g.sbo);
      constexpr uint64_t kStep = (2 * kLbo) >> 4;  // one K step: two core matrices
      const uint32_t acc_cols = (uint32_t)(g.n_rt * g.Npad);
      const int seg_ks = min(kc, L) / 16;
      const uint64_t rt_step = (uint64_t)((16u * g.sbo) >> 4);
      int acc = 0;
      uint32_t aph = 0;
      bool ok = true;
      for (long long i = 0; ok && i < n_chunks; i++) {
        const int s = (int)(i % nst);
        const uint32_t ph = (uint32_t)((i / nst) & 1);
        if (!tc::mbar_wait(&full[s], ph, abort_flag)) {
          raise();
          break;
        }
        tc::fence_after();
        const long long tc0 = ta + i * kc;
        const int n_ks = (int)min((long long)(kc / 16), (tb - tc0) / 16);
        uint64_t bd = desc0 + (uint64_t)(((uint32_t)s * g.stage_stride) >> 4);
        for (int j0 = 0; j0 < n_ks; j0 += seg_ks) {
          if (!tc::mbar_wait(&acce[acc], aph ^ 1, abort_flag)) {
            raise();
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t d = tmem + (uint32_t)acc * acc_cols;
          if (g.n_rt == 1) {
            for (int j = 0; j < seg_ks; j++, bd += kStep)
              tc::mma_bf16(d, bd, bd, idesc, j > 0 ? 1u : 0u);
          } else {
            for (int j = 0; j < seg_ks; j++, bd += kStep)
              for (int rt = 0; rt < g.n_rt; rt++)
                tc::mma_bf16(d + (uint32_t)(rt * g.Npad), bd + (uint64_t)rt * rt_step, bd, idesc,
                             j > 0 ? 1u : 0u);
          }
          tc::mma_commit(&accf[acc]);
          if (++acc == g.nacc) {
            acc = 0;
            aph ^= 1u;
          }
        }
        if (!ok) break;
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0, nullptr, 1u << 22);
    } else if (warp == kLoaderWarp) {
      // ------------------------------------------------------ loader
      // chunk i's antenna rows -> raw stage i % nraw, in chunk order, as far
      // ahead as the ring allows; before leaving, wait (bounded) for every
      // copy still in flight into this CTA's shared memory
      if (args.raw_path && lane == 0) {
        uint8_t* raw = smem + g.raw_off;
        long long issued = 0;
        for (long long i = 0; i < n_chunks; i++) {
          const int r = (int)(i % g.nraw);
          const uint32_t rph = (uint32_t)((i / g.nraw) & 1);
          if (!tc::mbar_wait(&raw_empty[r], rph ^ 1, abort_flag)) {
            raise();
            break;
          }
          const long long tc0 = ta + i * kc;
          const long long n_smp = min((long long)kc, tb - tc0);  // a multiple of 16
          const uint32_t bytes = (uint32_t)n_smp * 8u;
          tc::mbar_arrive_expect_tx(&raw_full[r], bytes * (uint32_t)M);
          for (int a = 0; a < M; a++)
            tc::bulk_g2s(raw + (size_t)r * g.raw_stride + (size_t)a * kc * 8,
                         args.y + (long long)a * args.n_samp + tc0, bytes, &raw_full[r]);
          issued = i + 1;
        }
        for (long long k = issued > g.nraw ? issued - g.nraw : 0; k < issued; k++)
          tc::mbar_wait(&raw_full[(int)(k % g.nraw)], (uint32_t)((k / g.nraw) & 1), nullptr,
                        1u << 22);
      }
    } else if (warp >= kEpiWarp0) {
      // ------------------------------------------------------ epilogue
      const int q = warp & 3;  // TMEM lane quarter of this warp
      const int n_pair = M * (M + 1) / 2;
      const int etid = threadIdx.x - 32 * kEpiWarp0;
      const uint32_t acc_cols = (uint32_t)(g.n_rt * g.Npad);
      const int ld = g.NC + 1;
      int acc = 0;
      uint32_t aph = 0;
      bool aborted = false;
      const int n_seg = L > kc ? L / kc : 1;  // accumulation segments per dump
      // up to 32 columns and one row tile: running sums in registers, stored
      // once per dump; lane quarters without used rows load nothing
      const bool reg_acc = g.n_rt == 1 && g.NC <= 32;
      const bool rows_used = 32 * q < g.KR;
      float racc[32];
      for (long long m = m_a; m < m_b; m++) {
        // each lane sums its own rows over the dump's segments
        for (int sg = 0; sg < n_seg; sg++) {
          if (!aborted && !tc::mbar_wait(&accf[acc], aph, abort_flag)) {
            raise();
            aborted = true;
          }
          tc::fence_after();
          if (!aborted && reg_acc) {
            if (rows_used) {
#pragma unroll
              for (int c0 = 0; c0 < 32; c0 += 16) {
                if (c0 >= g.NC) break;
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * acc_cols +
                                  (uint32_t)c0,
                              v);
#pragma unroll
                for (int c = 0; c < 16; c++) racc[c0 + c] = sg == 0 ? v[c] : racc[c0 + c] + v[c];
              }
            }
          } else if (!aborted) {
            for (int rt = 0; rt < g.n_rt; rt++) {
              const int row = rt * 128 + 32 * q + lane;
              for (int c0 = 0; c0 < g.NC; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * acc_cols +
                                  (uint32_t)(rt * g.Npad + c0),
                              v);
                if (row < g.KR)
#pragma unroll
                  for (int c = 0; c < 16; c++)
                    if (c0 + c < g.NC) {
                      float* d = &dsm[row * ld + c0 + c];
                      *d = sg == 0 ? v[c] : *d + v[c];
                    }
              }
            }
          }
          tc::fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&acce[acc]);
          if (++acc == g.nacc) {
            acc = 0;
            aph ^= 1u;
          }
        }
        if (reg_acc && !aborted && rows_used) {
          const int row = 32 * q + lane;
          if (row < g.KR)
#pragma unroll
            for (int c = 0; c < 32; c++)
              if (c < g.NC) dsm[row * ld + c] = racc[c];
        }
        // all four warps take the same stop decision
        uint32_t stop_u;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.ne.u32 p, %1, 0;\n\t"
            "bar.red.or.pred q, 1, 128, p;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(stop_u)
            : "r"((uint32_t)(aborted || *abort_flag != 0))
            : "memory");
        if (stop_u) break;
        float2* out = args.vis + m * n_pair;
        for (int p = etid; p < n_pair; p += 128) {
          int a = 0, r = p;
          while (r >= M - a) {
            r -= M - a;
            a++;
          }
          const int b = a + r;
          auto gm = [&](int k, int l) {
            float v = dsm[k * ld + l];
            if (args.terms == 3) v += dsm[(g.NC + k) * ld + l] + dsm[(g.NC + l) * ld + k];
            return v;
          };
          const float re = gm(2 * a, 2 * b) + gm(2 * a + 1, 2 * b + 1);
          const float im = gm(2 * a + 1, 2 * b) - gm(2 * a, 2 * b + 1);
          out[p] = make_float2(re, im);
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == kIssuerWarp) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

}  // namespace

bool corr_tc_supported(int n_ant, int dump_len, int terms) {
  CorrGeom g;
  return corr_geom(n_ant, terms, dump_len, &g);
}

cudaError_t launch_correlate_tc(const float2* y, long long n_samp, int n_ant, int dump_len,
                                long long first, long long last, float2* vis, int* err, int terms,
                                cudaStream_t st) {
  if (last < first) return cudaSuccess;
  CorrArgs a;
  if (!corr_geom(n_ant, terms, dump_len, &a.g)) return cudaErrorInvalidValue;
  // at least 116 KB so that a second CTA never shares the SM (and its TMEM)
  const uint32_t smem = a.g.total > 116 * 1024 ? a.g.total : 116 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_corr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const long long n_dumps = last - first + 1;
  long long grid = n_dumps < 152 ? n_dumps : 152;
  a.y = y;
  a.n_samp = n_samp;
  a.vis = vis;
  a.err = err;
  a.first = first;
  a.n_dumps = n_dumps;
  a.dumps_per_cta = (n_dumps + grid - 1) / grid;
  grid = (n_dumps + a.dumps_per_cta - 1) / a.dumps_per_cta;
  a.M = n_ant;
  a.L = dump_len;
  a.terms = terms;
  // bulk copies need 16-byte aligned rows: an even row length and base
  a.raw_path = a.g.nraw > 0 && (n_samp % 2) == 0 && ((uintptr_t)y % 16) == 0;
  k_corr_tc<<<(unsigned)grid, kCorrThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chirp
