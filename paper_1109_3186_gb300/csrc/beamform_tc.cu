// beamform_tc.cu -- Chimageator back-end on the tcgen05 tensor cores.
//
// Direct beamforming (Sec. 2.4.2) of the dedispersed voltages with
// narrowband weights W_pa = exp(+2 pi j f0 tau_a) (Eq. tau3D), detected and
// integrated per dump:  P[m][p] = sum_{t in dump m} |sum_a W_pa y_a(t)|^2.
//
// Complex GEMM in real-block form: row 2p gives Re b_p, row 2p+1 gives Im b_p,
//   A[2p  ][2a] =  Re W,  A[2p  ][2a+1] = -Im W,
//   A[2p+1][2a] =  Im W,  A[2p+1][2a+1] =  Re W,    B[2a + c][t] = (Re, Im)_c y_a(t),
// so D = A B holds the beams and P sums D^2 over both rows of a pixel.
//
// FP32 accuracy from BF16 tensor cores: every operand is split into a BF16
// head and a BF16 tail (x = x_h + x_l + O(2^-16 x)) and
//   D = A_h B_h + A_h B_l + A_l B_h    (A_l B_l is O(2^-16) and dropped).
// The three products are packed into ONE contraction: the K axis of the MMA
// walks [B_h | B_l | B_h] against [A_h | A_h | A_l], and because B_h and B_l
// sit next to each other in shared memory every 16-wide K step reads two
// adjacent 8-wide core-matrix columns.  For 12 antennas (24 real K) that is
// 72 useful of 80 MMA K (5 steps).
//
// Reduced-precision form (one term): the K axis holds only [B_h] against
// [A_h] (B tile padded to an even number of 8-wide k-groups with zeros), so
// 12 antennas take 3 MMA K steps instead of 5, with BF16 rounding of both
// operands (relative error ~2^-9 per product, FP32 accumulation).
//
// Layouts (no swizzle, K-major, 8-row x 16-byte core matrices):
//   A image per 128-row tile: [m-group 16][k-slot 2*ksteps][8 rows][8 bf16]
//     (K-major: a 16-byte row holds 8 K-values of one output row)
//   B tile of NT samples: [n-group NT/8][k-group GB][8 K-rows][8 samples bf16]
//     (MN-major: a 16-byte row holds 8 consecutive samples of one K-value,
//     which lets the inverse column pass write whole rows of one antenna)
//     three terms: GB = 2G, k-group g < G: heads of real K 8g..8g+7,
//     g >= G: tails of 8(g-G)...;  one term: GB = G rounded up to even, heads
//     only, the padding group zero.
//     real K index k = 2a + c (antenna a, c = 0 real / 1 imaginary).
// Both images are written in global memory in exactly this order so that one
// cp.async.bulk moves a whole tile.
//
// Kernel roles (320 threads): warp 0 lane 0 streams B tiles (bulk copies into
// a ring of 2-4 stages, as deep as shared memory allows); warp 1 owns TMEM (512 columns = 4 accumulators of 128) and
// its lane 0 issues the MMAs; warps 2-9 form two warpgroups that drain the
// accumulators of even / odd row tiles (one 128-column tcgen05.ld each), square
// and integrate per dump, and write whole-dump powers.  Every wait is bounded;
// on a timeout the kernel raises *err, drains its own copies and MMAs, frees
// TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tc.cuh"

namespace chirp {

namespace {

constexpr int RMAX = 8;        // row tiles per CTA (weights resident in smem)

// Bytes of one 128-row A tile with ks K-steps (16 row groups of 2 ks core
// matrices) and of one B tile of NT samples with GB k-groups.
__host__ __device__ constexpr uint32_t a_tile_bytes_of(int ks) {
  return 16u * 2u * (uint32_t)ks * 128u;
}
__host__ __device__ constexpr uint32_t b_tile_bytes_of(int NT, int GB) {
  return (uint32_t)(NT / 8) * (uint32_t)GB * 128u;
}

// Three shapes of the same kernel:
//  NT = 128, A in TMEM (AT): the weights are copied once into TMEM columns
//    256.. (128 lanes = rows, two BF16 per column) and every MMA reads A from
//    there, so shared memory feeds only B; 2 accumulators of 128 columns,
//    two warpgroups each draining the row tiles of one parity;
//  NT = 128 (any dump length): 4 accumulators of 128 columns, two warpgroups
//    each draining whole accumulators (row tiles of one parity);
//  NT = 256 (dump length a multiple of 256): 2 accumulators of 256 columns,
//    four warpgroups each draining a 64-column slice of every accumulator and
//    releasing it right after the load; the four partial sums of a row are
//    combined in shared memory once per dump.  The wider MMA halves the
//    shared-memory operand traffic per flop.
// MMA-issuing warps.  One thread can only issue so fast (each tcgen05.mma
// of a 128 x 256 x 16 tile, its descriptors, the per-row-tile barrier wait
// and commit); two warps, each owning the accumulators of one row-tile
// parity, keep the tensor pipe fed.
#ifndef CHIRP_BEAM_ISSUERS
#define CHIRP_BEAM_ISSUERS 2
#endif

template <int NT, bool AT = false>
struct BeamCfg {
  static_assert(!AT || NT == 128, "A in TMEM is used with 128-sample tiles");
  static constexpr int NACC = AT ? 2 : 512 / NT;  // TMEM accumulators
  static constexpr uint32_t A_COL = 256;          // AT: first TMEM column of the weights
  static constexpr int NSTAGE = NT == 256 ? 3 : 4;  // B ring depth (fewer when smem is short)
  static constexpr int EPI_WARPS = NT == 256 ? 16 : 8;
  static constexpr int ISSUERS = CHIRP_BEAM_ISSUERS;     // MMA-issuing warps
  static constexpr int EPI0 = 1 + ISSUERS;               // first epilogue warp
  static constexpr int THREADS = 32 * (EPI0 + EPI_WARPS);
  static constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, NT, true);  // B MN-major
  static constexpr uint32_t RED_BYTES = NT == 256 ? 4u * RMAX * 128u * 4u : 0u;
};

// Sum of squares of 64 values with paired FP32 FMAs (fma.rn.f32x2: two
// lanes per instruction), halving the epilogue's instruction count; four
// independent pair accumulators.
__device__ __forceinline__ float sumsq64(const float (&v)[64]) {
  unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
  for (int e = 0; e < 32; e++) {
    unsigned long long x;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(v[2 * e]), "f"(v[2 * e + 1]));
    asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc[e & 3]) : "l"(x));
  }
  float t = 0.f;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[j]));
    t += lo + hi;
  }
  return t;
}

struct BeamSmemPlan {
  uint32_t a_bytes, b_stage_bytes, red_off, bar_off, total;
};

template <int NT, bool AT = false>
__host__ __device__ inline BeamSmemPlan beam_smem_plan(int R, int ksteps, int G, int nstage) {
  BeamSmemPlan s;
  s.a_bytes = AT ? 0u : (uint32_t)R * a_tile_bytes_of(ksteps);
  s.b_stage_bytes = b_tile_bytes_of(NT, G);  // G here = k-groups per B tile
  s.red_off = s.a_bytes + (uint32_t)nstage * s.b_stage_bytes;
  s.bar_off = s.red_off + BeamCfg<NT, AT>::RED_BYTES;
  s.total = s.bar_off + 256;
  return s;
}

struct BeamArgs {
  const uint8_t* b_img;
  const uint8_t* a_img;
  float* pow;          // this DM: [n_dump][n_pix]
  int* err;
  long long t_begin;   // sample of column 0 of tile 0
  long long first;     // first valid dump
  long long n_dumps;   // valid dumps of this DM
  long long dumps_per_cta;
  int L, n_pix, n_rowtiles, R, GB, bwrap, ksteps;  // GB: k-groups per B tile
  int nstage;          // B ring depth, 2 .. BeamCfg<NT, AT>::NSTAGE
};

template <int NT, bool AT>
__global__ void __launch_bounds__(BeamCfg<NT, AT>::THREADS, 1) k_beam_tc(BeamArgs args) {
  using Cfg = BeamCfg<NT, AT>;
  constexpr int NACC = Cfg::NACC;
  constexpr int NSTAGE = Cfg::NSTAGE;  // barrier slots; the ring uses nst of them
  const int nst = args.nstage;
  constexpr uint32_t IDESC = Cfg::IDESC;
  extern __shared__ __align__(1024) uint8_t smem[];
  const BeamSmemPlan sp = beam_smem_plan<NT, AT>(args.R, args.ksteps, args.GB, nst);
  float* red = (float*)(smem + sp.red_off);  // NT = 256: [4 slices][RMAX][128 rows]
  uint8_t* smA = smem;
  uint8_t* smB = smem + sp.a_bytes;
  uint64_t* bars = (uint64_t*)(smem + sp.bar_off);
  static_assert(2 * NSTAGE + 2 * NACC + 2 <= 28, "barrier area");
  static_assert(NT == 128 || NT == 256, "tile width");
  static_assert(NACC % 2 == 0, "two draining warpgroups need an even accumulator count");
  uint64_t* full = bars;                 // [NSTAGE]
  uint64_t* empty = bars + NSTAGE;       // [NSTAGE]
  uint64_t* accf = bars + 2 * NSTAGE;    // [NACC]
  uint64_t* acce = accf + NACC;          // [NACC]
  uint64_t* abar = acce + NACC;          // A images
  uint64_t* drain = abar + 1;            // teardown of the MMA queue
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int rt0 = blockIdx.x * args.R;
  const int R_eff = min(args.R, args.n_rowtiles - rt0);
  // The pipeline always walks an even number of row tiles (a padding tile
  // is committed without MMAs and drained without reads).  Then accumulator
  // acc = u % NACC has the parity of r, so each accumulator -- and each of its
  // mbarriers -- has exactly one draining warpgroup, which can never be two
  // phases behind (phase parity would alias).
  const int R_pipe = (R_eff + 1) & ~1;
  // dumps of this CTA: [m_a, m_b) ; samples [ta, tb)
  const long long m_a = args.first + (long long)blockIdx.y * args.dumps_per_cta;
  const long long m_b = min(m_a + args.dumps_per_cta, args.first + args.n_dumps);
  const long long ta = m_a * args.L, tb = m_b * args.L;
  const long long j_a = (ta - args.t_begin) / NT;
  const long long j_b = (tb - args.t_begin + NT - 1) / NT;
  const long long n_tiles = (m_b > m_a && R_eff > 0) ? j_b - j_a : 0;
  const uint32_t a_tile_bytes = a_tile_bytes_of(args.ksteps);

  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; s++) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], Cfg::ISSUERS);  // every issuer commits once per tile
    }
    for (int a = 0; a < NACC; a++) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], NT == 256 ? 16 : 4);  // every draining warp arrives once
    }
    tc::mbar_init(abar, 1);
    tc::mbar_init(drain, Cfg::ISSUERS);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  if constexpr (AT) {
    // weights into TMEM: warpgroup wg copies the row tiles of its parity;
    // thread (quarter q, lane) holds row 32 q + lane of the tile
    if (warp >= Cfg::EPI0 && n_tiles > 0) {
      const int wg = (warp - Cfg::EPI0) / 4, q = warp & 3, row = 32 * q + lane;
      const int mg = row / 8, r8 = row % 8;
      for (int r = wg; r < R_eff; r += 2) {
        const uint8_t* src = args.a_img + (size_t)(rt0 + r) * a_tile_bytes +
                             (size_t)mg * (2 * args.ksteps * 128) + (size_t)r8 * 16;
        for (int ks = 0; ks < args.ksteps; ks++) {
          const uint4 lo = *reinterpret_cast<const uint4*>(src + (size_t)(2 * ks) * 128);
          const uint4 hi = *reinterpret_cast<const uint4*>(src + (size_t)(2 * ks + 1) * 128);
          const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
          tc::tmem_st8(tmem + ((uint32_t)(32 * q) << 16) + Cfg::A_COL +
                           (uint32_t)((r * args.ksteps + ks) * 8),
                       w);
        }
      }
      tc::tmem_wait_st();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }

  auto raise = [&]() {
    *abort_flag = 1;
    atomicExch(args.err, 1);
  };

  if (n_tiles > 0) {
    if (warp == 0 && lane == 0) {
      // ------------------------------------------------------ producer
      if constexpr (!AT) {
        tc::mbar_arrive_expect_tx(abar, (uint32_t)R_eff * a_tile_bytes);
        for (int r = 0; r < R_eff; r++)
          tc::bulk_g2s(smA + r * a_tile_bytes, args.a_img + (size_t)(rt0 + r) * a_tile_bytes,
                       a_tile_bytes, abar);
      }
      long long issued = 0;
      int s = 0;
      uint32_t ph = 0;
      for (long long i = 0; i < n_tiles; i++) {
        if (i > 0 && ++s == nst) {
          s = 0;
          ph ^= 1u;
        }
        if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
          raise();
          break;
        }
        tc::mbar_arrive_expect_tx(&full[s], sp.b_stage_bytes);
        tc::bulk_g2s(smB + (size_t)s * sp.b_stage_bytes,
                     args.b_img + (size_t)(j_a + i) * sp.b_stage_bytes, sp.b_stage_bytes,
                     &full[s]);
        issued = i + 1;
      }
      if (*abort_flag) {
        // let every copy this thread issued land before the CTA goes away
        if constexpr (!AT) tc::mbar_wait(abar, 0, nullptr, 1u << 22);
        for (long long i = issued > nst ? issued - nst : 0; i < issued; i++)
          tc::mbar_wait(&full[i % nst], (uint32_t)((i / nst) & 1), nullptr, 1u << 22);
      }
    } else if (warp >= 1 && warp <= Cfg::ISSUERS && lane == 0) {
      // ------------------------------------------------------ MMA issuers
      // Issuer `me` takes the row tiles r = me, me + ISSUERS, ... (and with
      // them the accumulators of that parity).  Descriptors are formed once
      // and advanced by adding the start-address offset (bytes / 16) of each
      // K step, stage and row tile.
      const int me = warp - 1;
      const uint32_t a_sbo = 2u * args.ksteps * 128u, b_sbo = (uint32_t)args.GB * 128u;
      const uint64_t a_desc0 = tc::sdesc(tc::smem_u32(smA), 128u, a_sbo);
      const uint64_t b_desc0 = tc::sdesc(tc::smem_u32(smB), 128u, b_sbo);
      const int ksteps = args.ksteps, bwrap = args.bwrap;
      bool ok = AT ? true : tc::mbar_wait(abar, 0, abort_flag);
      if (!ok) raise();
      int s = 0;
      uint32_t ph = 0;
      for (long long i = 0; ok && i < n_tiles; i++) {
        if (!tc::mbar_wait(&full[s], ph, abort_flag)) {
          raise();
          break;
        }
        tc::fence_after();
        const uint64_t b_desc = b_desc0 + (uint64_t)((s * sp.b_stage_bytes) >> 4);
        for (int r = me; r < R_pipe; r += Cfg::ISSUERS) {
          const unsigned long long u = (unsigned long long)(i * R_pipe + r);
          const int acc = (int)(u % NACC);
          const uint32_t aph = (uint32_t)((u / NACC) & 1);
          if (!tc::mbar_wait(&acce[acc], aph ^ 1, abort_flag)) {
            raise();
            ok = false;
            break;
          }
          tc::fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * NT);
          if (r < R_eff) {
            const uint64_t a_desc = a_desc0 + (uint64_t)((r * a_tile_bytes) >> 4);
            const uint32_t a_col = tmem + Cfg::A_COL + (uint32_t)(r * ksteps * 8);
            auto issue = [&](int ks) {
              const int p0 = 2 * ks;
              const int bg = p0 < bwrap ? p0 : p0 - bwrap;
              const uint64_t bd = b_desc + (uint64_t)(bg * 8);
              if constexpr (AT)
                tc::mma_bf16_ts(d, a_col + (uint32_t)(ks * 8), bd, IDESC, ks > 0 ? 1u : 0u);
              else
                tc::mma_bf16(d, a_desc + (uint64_t)(ks * 16), bd, IDESC, ks > 0 ? 1u : 0u);
            };
            // straight-line issue for the common K-step counts (12 antennas:
            // 5 split-BF16, 2 plain BF16 ... ), a loop otherwise
            switch (ksteps) {
              case 2: issue(0); issue(1); break;
              case 3: issue(0); issue(1); issue(2); break;
              case 5: issue(0); issue(1); issue(2); issue(3); issue(4); break;
              case 6: issue(0); issue(1); issue(2); issue(3); issue(4); issue(5); break;
              default:
                for (int ks = 0; ks < ksteps; ks++) issue(ks);
            }
          }
          tc::mma_commit(&accf[acc]);
        }
        if (!ok) break;
        tc::mma_commit(&empty[s]);
        if (++s == nst) {
          s = 0;
          ph ^= 1u;
        }
      }
      // nothing may be in flight when TMEM is released
      tc::mma_commit(drain);
      tc::mbar_wait(drain, 0, nullptr, 1u << 22);
    } else if (warp >= Cfg::EPI0) {
      if constexpr (NT == 256) {
        // ---------------------------------------------------- epilogue, 4 slices
        // Dumps start on tile boundaries (L % 256 == 0 and the CTA's range is
        // dump-aligned), so a dump ends only at the end of a tile.
        const int g = (warp - Cfg::EPI0) / 4;  // column slice [64 g, 64 g + 64)
        const int q = warp & 3;              // TMEM lane quarter of this warp
        const int row = 32 * q + lane;
        float sum[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; r++) sum[r] = 0.f;
        // No warp leaves the tile loop early: the per-dump combine uses a
        // named barrier, so after a timed-out wait this warp keeps walking
        // (later waits return at once because the abort flag is up) and all
        // warps leave together at the next combine point, or at the end.
        bool aborted = false;
        // counters instead of divisions: accumulator ring position, and the
        // tile within the current dump (dumps are whole tiles here)
        int acc = 0;
        uint32_t aph = 0;
        const int tiles_per_dump = args.L / NT;
        int tile_in_dump = 0;
        long long m = m_a;
        for (long long i = 0; i < n_tiles; i++) {
#pragma unroll
          for (int r = 0; r < RMAX; r++) {
            if (r >= R_pipe) break;
            if (!aborted && !tc::mbar_wait(&accf[acc], aph, abort_flag)) {
              raise();
              aborted = true;
            }
            tc::fence_after();
            float v[64];
            const bool use = !aborted && r < R_eff;
            if (use)
              tc::tmem_ld64(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * NT + 64 * g), v);
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[acc]);
            if (use) {
              sum[r] += sumsq64(v);
            }
            if (++acc == NACC) {
              acc = 0;
              aph ^= 1u;
            }
          }
          if (++tile_in_dump == tiles_per_dump) {  // this tile closes dump m (warp-uniform)
            tile_in_dump = 0;
#pragma unroll
            for (int r = 0; r < RMAX; r++) {
              if (r < R_eff) red[(g * RMAX + r) * 128 + row] = sum[r];
              sum[r] = 0.f;
            }
            // barrier with an OR of every epilogue thread's view of the abort
            // flag, so all warps take the same decision
            uint32_t stop_u;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\t"
                "setp.ne.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, 1, %2, p;\n\t"
                "selp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(stop_u)
                : "r"((uint32_t)(aborted || *abort_flag != 0)), "r"(32 * Cfg::EPI_WARPS)
                : "memory");
            const bool stop = stop_u != 0;
            if (!stop)
              for (int r = g; r < R_eff; r += 4) {
                float tot = 0.f;
#pragma unroll
                for (int gg = 0; gg < 4; gg++) tot += red[(gg * RMAX + r) * 128 + row];
                const float other = __shfl_xor_sync(0xffffffffu, tot, 1);
                const int p = ((rt0 + r) * 128 + row) >> 1;
                if (!(lane & 1) && p < args.n_pix) args.pow[m * args.n_pix + p] = tot + other;
              }
            asm volatile("bar.sync 1, %0;" ::"r"(32 * Cfg::EPI_WARPS) : "memory");
            if (stop) break;
            m++;
          }
        }
      } else {
      // ------------------------------------------------------ epilogue
      // warpgroup wg drains row tiles r = wg, wg + 2, ...; rr = r / 2 indexes
      // its per-row running dump sums.  All row tiles of a B tile cover the
      // same samples, so the dump boundary state (next_b) is per warpgroup.
      const int wg = (warp - Cfg::EPI0) / 4;
      const int q = warp & 3;              // TMEM lane quarter of this warp
      const int row = 32 * q + lane;       // row inside a 128-row tile
      constexpr int RH = RMAX / 2;
      float sum[RH];
#pragma unroll
      for (int rr = 0; rr < RH; rr++) sum[rr] = 0.f;
      long long next_b = ta + args.L;      // end of the dump being integrated
      auto flush = [&](int rr, long long m) {
        const float other = __shfl_xor_sync(0xffffffffu, sum[rr], 1);
        const int p = ((rt0 + 2 * rr + wg) * 128 + row) >> 1;
        if (!(lane & 1) && p < args.n_pix) args.pow[m * args.n_pix + p] = sum[rr] + other;
        sum[rr] = 0.f;
      };
      bool ok = true;
      for (long long i = 0; ok && i < n_tiles; i++) {
        const long long t0 = args.t_begin + (j_a + i) * NT;
        const long long tA = t0 > ta ? t0 : ta;
        const long long tB = (t0 + NT) < tb ? (t0 + NT) : tb;
        const bool clean = tA == t0 && tB == t0 + NT && t0 + NT <= next_b;  // warp-uniform
        long long nb_after = next_b;
#pragma unroll
        for (int rr = 0; rr < RH; rr++) {
          const int r = 2 * rr + wg;
          if (r >= R_pipe) break;
          const long long u = i * R_pipe + r;
          const int acc = (int)(u % NACC);
          const uint32_t aph = (uint32_t)((u / NACC) & 1);
          if (!tc::mbar_wait(&accf[acc], aph, abort_flag)) {
            raise();
            ok = false;
            break;
          }
          tc::fence_after();
          if (r >= R_eff) {  // padding tile: release without reading
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[acc]);
            continue;
          }
          const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * NT);
          if (clean) {
            float part = 0.f;
#pragma unroll
            for (int h = 0; h < NT / 64; h++) {
              float v[64];
              tc::tmem_ld64(tbase + 64 * h, v);
              part += sumsq64(v);
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[acc]);
            sum[rr] += part;
            if (t0 + NT == next_b) flush(rr, next_b / args.L - 1);
          } else {
            // tile at the edge of this CTA's range or holding a dump boundary
            long long nb = next_b;
#pragma unroll 1
            for (int c4 = 0; c4 < NT / 32; c4++) {
              const long long cs = t0 + 32 * c4;
              if (cs + 32 <= tA || cs >= tB) continue;  // warp-uniform
              float v[32];
              tc::tmem_ld32(tbase + 32 * c4, v);
              float part = 0.f;
#pragma unroll
              for (int e = 0; e < 32; e++) {
                const long long t = cs + e;  // warp-uniform
                if (t < tA || t >= tB) continue;
                part = fmaf(v[e], v[e], part);
                if (t + 1 == nb) {
                  sum[rr] += part;
                  part = 0.f;
                  flush(rr, nb / args.L - 1);
                  nb += args.L;
                }
              }
              sum[rr] += part;
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[acc]);
            nb_after = nb;
          }
        }
        if (clean) {
          if (t0 + NT == next_b) next_b += args.L;
        } else {
          next_b = nb_after;
        }
      }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

uint16_t bf16_bits_rn(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even (finite inputs)
  return (uint16_t)(u >> 16);
}
float bf16_to_float(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

}  // namespace

// A image (see the layout notes at the top) from FP64 weights W [n_pix][n_ant]
// given as interleaved (re, im).  Rows past 2 n_pix and antennas past n_ant
// are zero, as are the padding k-slots.  Slots: three terms [h h l 0],
// one term [h 0].
std::vector<uint8_t> build_beam_a_image(const double* W, int n_ant, int n_pix, int terms) {
  const int G = beam_tc_groups(n_ant), ks = beam_tc_ksteps(n_ant, terms);
  const int n_rowtiles = (2 * n_pix + 127) / 128;
  const size_t tile_bytes = a_tile_bytes_of(ks);
  std::vector<uint8_t> img((size_t)n_rowtiles * tile_bytes, 0);
  for (int rt = 0; rt < n_rowtiles; rt++)
    for (int mg = 0; mg < 16; mg++)
      for (int slot = 0; slot < 2 * ks; slot++) {
        int part, j;  // part 0 head, 1 tail, 2 zero
        if (slot < G) { part = 0; j = slot; }
        else if (terms == 1) { part = 2; j = 0; }
        else if (slot < 2 * G) { part = 0; j = slot - G; }
        else if (slot < 3 * G) { part = 1; j = slot - 2 * G; }
        else { part = 2; j = 0; }
        for (int r8 = 0; r8 < 8; r8++) {
          const int row = rt * 128 + mg * 8 + r8;
          const int p = row / 2, ri = row % 2;
          for (int e = 0; e < 8; e++) {
            const int k = 8 * j + e, a = k / 2, comp = k % 2;
            double v = 0.0;
            if (part != 2 && p < n_pix && a < n_ant) {
              const double wr = W[2 * ((size_t)p * n_ant + a)], wi = W[2 * ((size_t)p * n_ant + a) + 1];
              v = ri == 0 ? (comp == 0 ? wr : -wi) : (comp == 0 ? wi : wr);
            }
            const uint16_t h = bf16_bits_rn((float)v);
            const uint16_t bits = part == 0 ? h : bf16_bits_rn((float)(v - (double)bf16_to_float(h)));
            const size_t off = (size_t)rt * tile_bytes + (size_t)mg * (2 * ks * 128) +
                               (size_t)slot * 128 + (size_t)r8 * 16 + (size_t)e * 2;
            memcpy(&img[off], &bits, 2);
          }
        }
      }
  return img;
}

int beam_tc_groups(int n_ant) { return (n_ant + 3) / 4; }
int beam_tc_bgroups(int n_ant, int terms) {
  const int G = beam_tc_groups(n_ant);
  return terms == 3 ? 2 * G : (G + 1) & ~1;
}
int beam_tc_ksteps(int n_ant, int terms) {
  const int G = beam_tc_groups(n_ant);
  return terms == 3 ? (3 * G + 1) / 2 : (G + 1) / 2;
}
// Largest dynamic shared memory one CTA may request on sm_103 (227 KB).
constexpr uint32_t kSmemLimit = 227u * 1024u;

// Row tiles per CTA and B ring depth for a tile shape.  All CTA columns of
// a launch walk the same B tiles, so the column with the most row tiles sets
// the time: take the fewest columns that the largest fitting R allows (R
// fitting in 227 KB of shared memory with a 2-stage ring, and for AT its
// weights in the 256 TMEM columns beside the accumulators), spread the row
// tiles evenly over them, then use the deepest ring that still fits.  False
// when not even one row tile fits.
template <int NT, bool AT>
static bool beam_tc_shape(int ks, int GB, int n_rowtiles, int* R_out, int* nst_out) {
  auto fits = [&](int R, int nst) {
    if (AT && R * ks * 8 > 512 - (int)BeamCfg<NT, AT>::A_COL) return false;
    return beam_smem_plan<NT, AT>(R, ks, GB, nst).total <= kSmemLimit;
  };
  int rmax = 0;
  for (int R = RMAX < n_rowtiles ? RMAX : n_rowtiles; R >= 1 && !rmax; R--)
    if (fits(R, 2)) rmax = R;
  if (!rmax) return false;
  const int gx = (n_rowtiles + rmax - 1) / rmax;
  const int R = (n_rowtiles + gx - 1) / gx;
  int nst = 2;
  for (int s = BeamCfg<NT, AT>::NSTAGE; s > 2; s--)
    if (fits(R, s)) {
      nst = s;
      break;
    }
  *R_out = R;
  *nst_out = nst;
  return true;
}

// Kernel shape for a search: 0 none fits, 1 = 128-sample tiles with the
// weights in shared memory, 2 = 256-sample tiles (dump length a multiple of
// 256), 3 = 128-sample tiles with the weights in TMEM.  Preference, from
// timing the 12-antenna, 1024-beam search (beam stage per 64 DMs): 2 (84.6
// ms), then 1 (131 ms), then 3 (150 ms; it only frees shared memory, which
// matters when the weights of one row tile do not fit there).

int beam_tc_pick(int n_ant, int n_pix, int dump_len, int terms, int forced) {
  const int ks = beam_tc_ksteps(n_ant, terms), GB = beam_tc_bgroups(n_ant, terms);
  const int n_rowtiles = (2 * n_pix + 127) / 128;
  int R, nst;
  const bool at = beam_tc_shape<128, true>(ks, GB, n_rowtiles, &R, &nst);
  const bool w256 = dump_len % 256 == 0 && beam_tc_shape<256, false>(ks, GB, n_rowtiles, &R, &nst);
  const bool w128 = beam_tc_shape<128, false>(ks, GB, n_rowtiles, &R, &nst);
  if (forced != 0)
    return (forced == 3 && at) || (forced == 2 && w256) || (forced == 1 && w128) ? forced : 0;
  if (w256) return 2;
  if (w128) return 1;
  if (at) return 3;
  return 0;
}


int beam_tc_tile_samples(int shape) { return shape == 0 ? 0 : (shape == 2 ? 256 : 128); }
long long beam_tc_tile_bytes(int n_ant, int shape, int terms) {
  const int nt = beam_tc_tile_samples(shape);
  return nt ? (long long)b_tile_bytes_of(nt, beam_tc_bgroups(n_ant, terms)) : 0;
}


namespace {

template <int NT, bool AT>
static cudaError_t launch_beam_tc_nt(const uint8_t* b_img, const uint8_t* a_img, int n_ant,
                                     int n_pix, int dump_len, long long first, long long last,
                                     long long t_origin, float* pow, int* err, int terms,
                                     cudaStream_t st) {
  using Cfg = BeamCfg<NT, AT>;
  const int ks = beam_tc_ksteps(n_ant, terms), G = beam_tc_bgroups(n_ant, terms);
  const int n_rowtiles = (2 * n_pix + 127) / 128;
  int R, nst;
  if (!beam_tc_shape<NT, AT>(ks, G, n_rowtiles, &R, &nst)) return cudaErrorInvalidConfiguration;
  const BeamSmemPlan sp = beam_smem_plan<NT, AT>(R, ks, G, nst);
  // at least 116 KB so that a second CTA never shares the SM (and its TMEM)
  const uint32_t smem_bytes = sp.total > 116 * 1024 ? sp.total : 116 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_beam_tc<NT, AT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  const int gx = (n_rowtiles + R - 1) / R;
  const long long n_dumps = last - first + 1;
  long long gy = (152 + gx - 1) / gx;  // about one CTA per SM
  if (gy > n_dumps) gy = n_dumps;
  if (gy < 1) gy = 1;
  BeamArgs a;
  a.b_img = b_img;
  a.a_img = a_img;
  a.pow = pow;
  a.err = err;
  a.t_begin = t_origin;
  a.first = first;
  a.n_dumps = n_dumps;
  a.dumps_per_cta = (n_dumps + gy - 1) / gy;
  gy = (n_dumps + a.dumps_per_cta - 1) / a.dumps_per_cta;
  a.L = dump_len;
  a.n_pix = n_pix;
  a.n_rowtiles = n_rowtiles;
  a.R = R;
  a.GB = G;
  a.bwrap = terms == 3 ? 2 * beam_tc_groups(n_ant) : G;
  a.ksteps = ks;
  a.nstage = nst;
  k_beam_tc<NT, AT><<<dim3(gx, (unsigned)gy), Cfg::THREADS, smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_beam_tc(const uint8_t* b_img, const uint8_t* a_img, int n_ant, int n_pix,
                           int dump_len, long long first, long long last, long long t_origin,
                           float* pow, int* err, int terms, int shape, cudaStream_t st) {
  if (last < first) return cudaSuccess;
  if (t_origin > first * dump_len) return cudaErrorInvalidValue;
  if (shape == 2 && (first * dump_len - t_origin) % 256) return cudaErrorInvalidValue;
  switch (shape) {
    case 3:
      return launch_beam_tc_nt<128, true>(b_img, a_img, n_ant, n_pix, dump_len, first, last,
                                          t_origin, pow, err, terms, st);
    case 2:
      return launch_beam_tc_nt<256, false>(b_img, a_img, n_ant, n_pix, dump_len, first, last,
                                           t_origin, pow, err, terms, st);
    case 1:
      return launch_beam_tc_nt<128, false>(b_img, a_img, n_ant, n_pix, dump_len, first, last,
                                           t_origin, pow, err, terms, st);
    default:
      return cudaErrorInvalidConfiguration;
  }
}

}  // namespace chirp
