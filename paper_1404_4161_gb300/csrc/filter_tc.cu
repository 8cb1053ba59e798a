// Split-precision Chebyshev filter on the GB300 tensor cores (tcgen05 +
// TMEM + TMA), sm_103a: every step of Alg. 2 for one or many problems in
// ONE persistent cooperative launch.
//
// Each step of the Alg. 2 recurrence computes Y_{i+1} = a_i (H Y_i - c Y_i) +
// b_i Y_{i-1} on the active (still unfinished) suffix of the degree-sorted
// block.  The complex product is one real GEMM
//
//     [Hr | Hi] (n x 2n)  *  B (2n x 2k)  ->  [.. Zr_j, Zi_j ..] (n x 2k)
//
// with B's columns interleaved per complex column j: column 2j holds
// (Yr_j ; -Yi_j) and column 2j+1 holds (Yi_j ; Yr_j), so the real and
// imaginary parts of each output element sit in adjacent accumulator
// columns.  A = [Hr | Hi] is built once per problem (row r of A is the
// conjugate of column r of the Hermitian H, read contiguously).
//
// Split formats: every operand x is cut into bf16 pieces x = x0 + x1 + x2,
// x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1).  With two pieces
// the product keeps x0 y0 + x0 y1 + x1 y0 (3 products, ~2^-16 relative);
// with three it adds x0 y2 + x1 y1 + x2 y0 (6 products, ~2^-23 for the
// split).  The tensor cores accumulate in FP32 rounding toward zero (a
// bias of about 0.3 ulp of the running sum per accumulate, measured: -3e-5
// relative after the 1536 accumulates of one 3-product tile at n = 4096),
// so every tile is accumulated in K chunks of 512 (3 products) or 256 (6
// products) whose partial sums the epilogue adds in FP32 registers, the
// leading product x0 y0 in an accumulator of its own.
//
// "Defect" form (iterative refinement of the filter, not in the paper):
// for vectors Y with a diagonal of shifts Lambda (Ritz values) and R = HY -
// Y Lambda, the filtered block is p(H) Y = Y psi(Lambda) + D, where psi is
// the scalar recurrence applied to each shift and D follows the same
// three-term recurrence driven by R:
//     D_0 = 0,  D_1 = a_0 R,
//     D_{i+1} = a_i (H D_i - c D_i) + b_i D_{i-1} + a_i psi_i(lambda_j) R_j.
// D is of the size of the residual, so computing it in split precision
// leaves an error of (split precision) x (residual) instead of the split
// precision itself; Y psi(Lambda) is formed in FP64.
//
// Work decomposition (one launch per filter call):
//   * A "segment" is one step of one problem; segments are ordered by
//     (step, problem).  The columns of a problem are cut into blocks of N
//     real columns at fixed positions (block b = columns [bN, (b+1)N)); a
//     segment's tiles are (block, row tile) pairs and a tile covers the
//     part of its block that is still active at that step.  Blocks are
//     taken in groups of up to (SMs / row tiles), row-tile-major inside a
//     group, so that the tiles sharing a row tile of A run side by side and
//     read it from L2 once.
//   * Output tile (m, b) of step i+1 reads the whole of Y_i's block b, so
//     it waits until every row tile of block b of step i is published (a
//     per-(segment, block) counter).  Steps therefore overlap: the blocks
//     of step i+1 start while later blocks of step i still run, and no
//     wave of a step waits for the slowest tile of the previous one.
//   * CTA g (one per SM, all co-resident under the cooperative launch)
//     takes tiles g, g + G, g + 2G, ... in increasing order; a tile only
//     waits on tiles of earlier segments, which have smaller indices, so
//     the smallest unfinished tile never waits and every wait ends.  Each
//     wait is still bounded (globaltimer) and watches a global abort word.
// Inside a CTA (256 threads):
//   warp 0 lane 0: TMA producer (A pieces, B pieces per 64-wide K block)
//   warp 1 lane 0: tcgen05.mma issuer; chunk g of the CTA's tiles goes to
//                  TMEM slot g % 2 (2 slots x 2 accumulators x 128 columns)
//   warp 2:        TMEM allocation / release
//   warps 4-7:     epilogue: drain every chunk (tcgen05.ld) into FP32
//                  registers, which overlaps the MMAs of the next chunks;
//                  after a tile's last chunk the recurrence -> FP32 master
//                  of Y_{i+1}, bf16 pieces of the next B operand, FP64
//                  output of the columns that finish at this step; then the
//                  tile is published: generic stores -> fence.proxy.async
//                  (the next step reads them with TMA) -> the last epilogue
//                  warp's release add on the (segment, block) counter.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int MAX_PIECES = 3;

struct FProb {
  int n, k, P, kblocks, ntile;
  float2* M;           // three FP32 masters, n x k each
  __nv_bfloat16* B;    // [buf][piece] blocks of 2k x P
  long long b_elems;   // 2k * P
  double2* out;        // FP64 output, n x k
  const float2* Rf;    // forcing block of the refinement form (FP32), or null
};

struct FSeg {
  int p, step, tile_base, mt, blk0, nblk;
  int grp;              // blocks per tile group (row-tile-major inside a group)
  int s_col, s_new;     // first active column; columns below s_new finish here
  float a, b, c;
  int cur, prev, next;  // master indices; prev < 0 when b == 0
  int bin, bout;        // B buffers read / written
  int dep, dep_blk0, dep_done;  // previous segment of the problem (-1: none)
  int done_base;        // counters of this segment's blocks
  const double* fR;     // forcing coefficients of this step (k doubles) or null
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until *cnt >= target; false on timeout or global abort.
__device__ bool wait_count(const int* cnt, int target, volatile int* abort_g, int* err) {
  if (ld_acquire(cnt) >= target) return true;
  const unsigned long long t0 = globaltimer();
  while (ld_acquire(cnt) < target) {
    if (*abort_g) return false;
    if (globaltimer() - t0 > WAIT_NS) {
      *abort_g = 1;
      atomicExch(err, 4);
      return false;
    }
  }
  return true;
}

// Bounded mbarrier wait that also watches the global abort word.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_sh,
                                         volatile int* abort_g, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_sh || *abort_g) return false;
    if (globaltimer() - t0 > WAIT_NS) {
      *abort_sh = 1;
      *abort_g = 1;
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ int find_seg(const FSeg* segs, int nsegs, int t) {
  int lo = 0, hi = nsegs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct TileGeo {
  int m0, bi, cs, ce;  // row start, block within the segment, real column range [cs, ce)
};
// Tiles of a segment: blocks in groups of sg.grp; inside a group, row tile
// major (the blocks of one row tile are consecutive, so the CTAs holding
// them run side by side and read the same A K blocks from L2).
__device__ __forceinline__ TileGeo tile_geo(const FSeg& sg, const FProb& pr, int t) {
  TileGeo g;
  const int local = t - sg.tile_base;
  const int gi = local / (sg.mt * sg.grp);
  const int rem = local - gi * sg.mt * sg.grp;
  const int gsz = min(sg.grp, sg.nblk - gi * sg.grp);
  g.bi = gi * sg.grp + rem % gsz;
  g.m0 = (rem / gsz) * BM;
  const int b = sg.blk0 + g.bi;
  g.cs = max(b * pr.ntile, 2 * sg.s_col);
  g.ce = min((b + 1) * pr.ntile, 2 * pr.k);
  return g;
}

__device__ __forceinline__ void split_pieces(float x, __nv_bfloat16 (&q)[MAX_PIECES]) {
  q[0] = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(q[0]);
  q[1] = __float2bfloat16_rn(r1);
  q[2] = __float2bfloat16_rn(r1 - __bfloat162float(q[1]));
}

// Accumulator slots: TMEM (512 columns) holds RING = 2 slots.  A tile's K
// range is cut into chunks of KCfg::KB K blocks; chunk g (counted over all
// tiles of the CTA) accumulates into slot g % RING and is drained by the
// epilogue warps into FP32 registers (round-to-nearest adds).  The tensor
// cores' FP32 accumulation rounds toward zero (a bias of about 0.3 ulp of
// the running sum per accumulate); draining every chunk bounds that bias by
// the chunk's accumulates instead of the whole K range.
//   * Three products (NS = 2): one accumulator of up to 256 columns per slot
//     (a 128 x 256 output tile); the chunk's 96 accumulates leave a bias
//     of about 2e-6 of the chunk sum, within the format's 2^-16.  Sixteen
//     epilogue warps, four per TMEM lane quarter, 64 columns each.
//   * Six products (NS = 3): two accumulators of 128 columns per slot, the
//     leading product x0 y0 in the first (its sum sees one accumulate per 16
//     of K) and the smaller products in the second (their bias is relative
//     to their own, 2^-8 smaller, sum).  Eight epilogue warps, two per TMEM
//     lane quarter, 64 columns each.
constexpr int RING = 2;
template <int NS>
struct KCfg;
template <>
struct KCfg<2> {
  static constexpr int SLOT = 256;  // accumulator columns
  static constexpr int NACC = 1;    // accumulators per slot
  static constexpr int EPW = 16;    // epilogue warps
  static constexpr int KB = 8;      // K blocks (64 wide) per chunk
  static constexpr int EP_GRP = 1;  // complex columns per batch of the epilogue's loads
};
template <>
struct KCfg<3> {
  static constexpr int SLOT = 128;
  static constexpr int NACC = 2;
  static constexpr int EPW = 8;
  static constexpr int KB = 4;
  static constexpr int EP_GRP = 2;
};
template <int NS>
constexpr int kthreads() {
  return 128 + 32 * KCfg<NS>::EPW;
}

template <int NS>
__global__ void __launch_bounds__(kthreads<NS>(), 1)
tc_filter_kernel(const FProb* __restrict__ probs, const FSeg* __restrict__ segs, int nsegs,
                 int total_tiles, const CUtensorMap* __restrict__ maps, int nmax, int stages,
                 int* done, int* abort_g_ptr, int* err) {
  constexpr int CKB = KCfg<NS>::KB;
  constexpr int EP_GRP = KCfg<NS>::EP_GRP;
  constexpr int SLOT = KCfg<NS>::SLOT;
  constexpr int NACC = KCfg<NS>::NACC;
  constexpr int EPW = KCfg<NS>::EPW;
  constexpr int CW = SLOT * 4 / EPW;  // accumulator columns per epilogue thread
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t bmax_bytes = (uint32_t)nmax * BK * 2;
  const uint32_t stage_bytes = NS * (a_bytes + bmax_bytes);
  uint64_t* bars = (uint64_t*)(smem + (size_t)stages * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* sfull = bars + 2 * stages;  // [RING]
  uint64_t* sempty = sfull + RING;      // [RING], EPW arrivals (epilogue warps)
  uint64_t* fin = sempty + RING;        // MMA completion before TMEM release
  uint32_t* tmem_slot = (uint32_t*)(fin + 1);
  volatile int* abort_sh = (volatile int*)(tmem_slot + 1);
  int* ep_count = (int*)(tmem_slot + 2);  // [8]: per-tile arrivals of the epilogue warps
  volatile int* abort_g = (volatile int*)abort_g_ptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(&sfull[r], 1);
      mbar_init(&sempty[r], EPW);
    }
    mbar_init(fin, 1);
    for (int i = 0; i < 8; ++i) ep_count[i] = 0;
    *abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) tmem_alloc(tmem_slot, RING * NACC * SLOT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    uint32_t kbg = 0;
    int issued_lo = 0, issued_hi = 0;  // kbg range of the last stages armed
    for (int t = blockIdx.x; t < total_tiles && !*abort_g; t += gridDim.x) {
      const FSeg& sg = segs[find_seg(segs, nsegs, t)];
      const FProb& pr = probs[sg.p];
      const TileGeo g = tile_geo(sg, pr, t);
      if (sg.dep >= 0 && !wait_count(done + sg.dep_done + (sg.blk0 + g.bi - sg.dep_blk0), sg.mt,
                                     abort_g, err))
        break;
      fence_proxy_async_global();
      const CUtensorMap* mp = maps + (size_t)sg.p * 9;
      const uint32_t bytes = NS * (a_bytes + (uint32_t)pr.ntile * BK * 2);
      bool ok = true;
      for (int kb = 0; kb < pr.kblocks; ++kb, ++kbg) {
        const int s = (int)(kbg % (uint32_t)stages);
        const uint32_t ph = (kbg / (uint32_t)stages) & 1u;
        if (!wait_bar(&empty[s], ph ^ 1u, abort_sh, abort_g, err, 5)) {
          ok = false;
          break;
        }
        unsigned char* st = smem + (size_t)s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
        for (int q = 0; q < NS; ++q)
          tma_load_2d(st + q * a_bytes, mp + q, &full[s], kb * BK, g.m0);
#pragma unroll
        for (int q = 0; q < NS; ++q)
          tma_load_2d(st + NS * a_bytes + q * bmax_bytes, mp + 3 + 3 * sg.bin + q, &full[s],
                      kb * BK, g.cs);
        issued_hi = (int)kbg + 1;
        issued_lo = issued_hi > stages ? issued_hi - stages : 0;
      }
      if (!ok) break;
    }
    if (*abort_sh || *abort_g) {
      // let the copies still in flight land before shared memory is released
      for (int kb = issued_lo; kb < issued_hi; ++kb) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full[kb % stages], (uint32_t)(kb / stages) & 1u) &&
               globaltimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    uint32_t kbg = 0, gch = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total_tiles && ok; t += gridDim.x) {
      const FSeg& sg = segs[find_seg(segs, nsegs, t)];
      const FProb& pr = probs[sg.p];
      const TileGeo g = tile_geo(sg, pr, t);
      const int nmma = (g.ce - g.cs + 15) / 16 * 16;
      const uint32_t idesc = idesc_bf16(BM, nmma);
      for (int kc = 0; kc < pr.kblocks && ok; kc += CKB, ++gch) {
        const int slot = (int)(gch % RING);
        if (!wait_bar(&sempty[slot], ((gch / RING) & 1u) ^ 1u, abort_sh, abort_g, err, 6)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d_lead = tmem + (uint32_t)(slot * NACC * SLOT);
        const uint32_t d_tail = NACC == 2 ? d_lead + SLOT : d_lead;
        const int kend = min(pr.kblocks, kc + CKB);
        for (int kb = kc; kb < kend; ++kb, ++kbg) {
          const int s = (int)(kbg % (uint32_t)stages);
          const uint32_t ph = (kbg / (uint32_t)stages) & 1u;
          if (!wait_bar(&full[s], ph, abort_sh, abort_g, err, 7)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
          const uint32_t sb = sa + NS * a_bytes;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 16 bf16 = 32 B along K
            const uint32_t acc0 = (kb > kc || kk > 0) ? 1u : 0u;
            // pieces (qa, qb) with qa + qb <= NS - 1: the leading product
            // into the lead accumulator, the others into the tail one
            umma_bf16(d_lead, desc_sw128(sa) + adv, desc_sw128(sb) + adv, idesc, acc0);
#pragma unroll
            for (int ssum = 1; ssum < NS; ++ssum) {
#pragma unroll
              for (int qa = 0; qa <= ssum; ++qa) {
                const int qb = ssum - qa;
                // one shared accumulator: only the leading product starts it
                umma_bf16(d_tail, desc_sw128(sa + qa * a_bytes) + adv,
                          desc_sw128(sb + qb * bmax_bytes) + adv, idesc,
                          (NACC == 2 && ssum == 1 && qa == 0) ? acc0 : 1u);
              }
            }
          }
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&sfull[slot]);
      }
    }
    // every MMA issued so far completes before the TMEM is released
    umma_commit(fin);
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(fin, 0u) && globaltimer() - t0 < WAIT_NS) {
    }
  } else if (warp >= 4) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    const int col0 = ((warp - 4) >> 2) * CW;  // this warp's columns [col0, col0 + CW)
    uint32_t tc = 0, gch = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++tc) {
      const int si = find_seg(segs, nsegs, t);
      const FSeg& sg = segs[si];
      const FProb& pr = probs[sg.p];
      const TileGeo g = tile_geo(sg, pr, t);
      const int width = g.ce - g.cs - col0;
      float acc[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) acc[c] = 0.f;
      bool ok = true;
      for (int kc = 0; kc < pr.kblocks; kc += CKB, ++gch) {
        const int slot = (int)(gch % RING);
        if (!wait_bar(&sfull[slot], (gch / RING) & 1u, abort_sh, abort_g, err, 8)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tq =
            tmem + (uint32_t)(slot * NACC * SLOT + col0) + ((uint32_t)(q * 32) << 16);
#pragma unroll
        for (int c0 = 0; c0 < CW; c0 += 16) {
          if (c0 < width) {  // uniform across the warp
            float v[16];
            __syncwarp();
            tmem_ld16(tq + (uint32_t)c0, v);  // warp-collective
            if (NACC == 2) {
              float w[16];
              tmem_ld16(tq + (uint32_t)(SLOT + c0), w);
#pragma unroll
              for (int c = 0; c < 16; ++c) acc[c0 + c] += v[c] + w[c];
            } else {
#pragma unroll
              for (int c = 0; c < 16; ++c) acc[c0 + c] += v[c];
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sempty[slot]);
      }
      if (!ok) break;
      if (sg.dep >= 0)  // orders the master reads below after the producers' stores
        (void)ld_acquire(done + sg.dep_done + (sg.blk0 + g.bi - sg.dep_blk0));
      const int row = g.m0 + q * 32 + lane;
      if (row < pr.n) {
        const int n = pr.n, k = pr.k;
        const size_t nk = (size_t)n * k;
        const float2* cur = pr.M + (size_t)sg.cur * nk;
        const float2* prev = sg.prev >= 0 ? pr.M + (size_t)sg.prev * nk : nullptr;
        float2* next = pr.M + (size_t)sg.next * nk;
        const float2* Rf = sg.fR ? pr.Rf : nullptr;
        __nv_bfloat16* bo = pr.B + (size_t)(3 * sg.bout) * pr.b_elems;
        // columns in batches of EP_GRP: the batch's loads are issued
        // together (L2, coherent with the other SMs' stores), then the
        // recurrence and the stores, so a tile pays a few L2 latencies
        // instead of one per column
#pragma unroll
        for (int cb = 0; cb < CW; cb += 2 * EP_GRP) {
          if (g.cs + col0 + cb >= g.ce) continue;  // uniform across the warp
          float2 cu[EP_GRP], pv[EP_GRP], rr[EP_GRP];
          float fr[EP_GRP];
#pragma unroll
          for (int u = 0; u < EP_GRP; ++u) {
            const int rc = g.cs + col0 + cb + 2 * u;
            cu[u] = pv[u] = rr[u] = make_float2(0.f, 0.f);
            fr[u] = 0.f;
            if (rc < g.ce) {
              const int j = rc >> 1;
              const size_t e = (size_t)row + (size_t)j * n;
              cu[u] = __ldcg(cur + e);
              if (prev) pv[u] = __ldcg(prev + e);
              if (Rf) {
                rr[u] = __ldcg(Rf + e);
                fr[u] = (float)__ldg(sg.fR + j);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < EP_GRP; ++u) {
            const int c2 = cb + 2 * u;  // index into acc
            const int rc = g.cs + col0 + c2;  // real column (even)
            if (rc < g.ce) {
              const int j = rc >> 1;  // complex column
              const size_t e = (size_t)row + (size_t)j * n;
              float re = sg.a * (acc[c2] - sg.c * cu[u].x);
              float im = sg.a * (acc[c2 + 1] - sg.c * cu[u].y);
              if (prev) {
                re = fmaf(sg.b, pv[u].x, re);
                im = fmaf(sg.b, pv[u].y, im);
              }
              if (Rf) {
                re = fmaf(fr[u], rr[u].x, re);
                im = fmaf(fr[u], rr[u].y, im);
              }
              next[e] = make_float2(re, im);
              __nv_bfloat16 pre[MAX_PIECES], pim[MAX_PIECES], pnim[MAX_PIECES];
              split_pieces(re, pre);
              split_pieces(im, pim);
              split_pieces(-im, pnim);
              const size_t r0 = (size_t)(2 * j) * pr.P, r1 = r0 + pr.P;
#pragma unroll
              for (int pc = 0; pc < NS; ++pc) {
                __nv_bfloat16* bq = bo + (size_t)pc * pr.b_elems;
                bq[r0 + row] = pre[pc];       // column 2j, top:      Yr
                bq[r1 + n + row] = pre[pc];   // column 2j+1, bottom: Yr
                bq[r1 + row] = pim[pc];       // column 2j+1, top:    Yi
                bq[r0 + n + row] = pnim[pc];  // column 2j, bottom:   -Yi
              }
              if (j < sg.s_new) pr.out[e] = make_double2((double)re, (double)im);
            }
          }
        }
      }
      // The last of the epilogue warps to finish this tile publishes it
      // (no CTA barrier, so an aborting warp cannot block the others).  A
      // warp is at most RING tiles ahead of the slowest one (each tile takes
      // at least one slot), so 8 per-tile counters are never shared.
      fence_proxy_async_global();
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        const int arrived = atomicAdd(&ep_count[tc & 7u], 1);
        if (arrived == EPW * (int)(tc >> 3) + EPW - 1) {
          __threadfence();
          red_release_add(done + sg.done_base + g.bi, 1);
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, RING * NACC * SLOT);
  }
}

// ------------------------------------------------- operand preparation --
// Row r of A = [Re H[r, :] | Im H[r, :]] in `pieces` bf16 pieces; for
// Hermitian H, H[r, x] = conj(H[x, r]), so row r is read from column r
// (contiguous).
__global__ void repack_h_kernel(int n, int P, int pieces, const double2* __restrict__ H,
                                __nv_bfloat16* __restrict__ A, size_t a_elems) {
  const int r = blockIdx.y;
  const double2* col = H + (size_t)r * n;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < 2 * n; x += gridDim.x * blockDim.x) {
    double v = (x < n) ? col[x].x : -col[x - n].y;
    for (int q = 0; q < pieces; ++q) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      A[(size_t)q * a_elems + (size_t)r * P + x] = h;
      v -= (double)__bfloat162float(h);
    }
  }
}

// B operand pieces (buffer `bout`) + FP32 master of an n x k block.  Plain
// form: src = Y0 (scale 1).  Defect form: src = R, scale = a_0 (D_1 = a_0
// R).  Columns below fin_end are also written to out (FP64) when out is
// not null.  Rf (when not null) receives src in FP32, unscaled.
__global__ void split_block_kernel(int n, int k, int P, const double2* __restrict__ src,
                                   double scale, float2* __restrict__ master,
                                   __nv_bfloat16* __restrict__ B, size_t b_elems,
                                   double2* __restrict__ out, int fin_end,
                                   float2* __restrict__ Rf) {
  const int j = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const size_t e = (size_t)r + (size_t)j * n;
    const double2 s = src[e];
    if (Rf) Rf[e] = make_float2((float)s.x, (float)s.y);
    const float re = (float)(scale * s.x), im = (float)(scale * s.y);
    master[e] = make_float2(re, im);
    if (out && j < fin_end) out[e] = make_double2(scale * s.x, scale * s.y);
    __nv_bfloat16 pre[MAX_PIECES], pim[MAX_PIECES], pnim[MAX_PIECES];
    split_pieces(re, pre);
    split_pieces(im, pim);
    split_pieces(-im, pnim);
    const size_t r0 = (size_t)(2 * j) * P, r1 = r0 + P;
#pragma unroll
    for (int pc = 0; pc < MAX_PIECES; ++pc) {
      __nv_bfloat16* bq = B + (size_t)pc * b_elems;
      bq[r0 + r] = pre[pc];
      bq[r1 + n + r] = pre[pc];
      bq[r1 + r] = pim[pc];
      bq[r0 + n + r] = pnim[pc];
    }
  }
}

// psi[i * k + j] = psi_i(lambda_j): the filter's scalar recurrence on each
// shift (psi_0 = 1, psi_1 = a_0 (lambda - c), psi_{i+1} = a_i (lambda - c)
// psi_i + b_i psi_{i-1}).  coef = {a_0, (a_i, b_i) for i >= 1}.
__global__ void psi_table_kernel(int k, int m, const double* __restrict__ lam, double c,
                                 const double* __restrict__ coef, double* __restrict__ psi) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const double t = lam[j] - c;
  double p0 = 1.0, p1 = coef[0] * t;
  psi[j] = p0;
  if (m >= 1) psi[(size_t)k + j] = p1;
  for (int i = 1; i < m; ++i) {
    const double p2 = coef[2 * i - 1] * t * p1 + coef[2 * i] * p0;
    psi[(size_t)(i + 1) * k + j] = p2;
    p0 = p1;
    p1 = p2;
  }
}

// Y'_j = Y_j psi_{m_j}(lambda_j) + D_j (FP64), in place on D.
__global__ void defect_combine_kernel(int n, int k, const double2* __restrict__ Y,
                                      const int* __restrict__ deg, const double* __restrict__ psi,
                                      double2* __restrict__ D) {
  const int j = blockIdx.y;
  const double f = psi[(size_t)deg[j] * k + j];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const size_t e = (size_t)r + (size_t)j * n;
    const double2 y = Y[e];
    double2 d = D[e];
    d.x = fma(f, y.x, d.x);
    d.y = fma(f, y.y, d.y);
    D[e] = d;
  }
}

// out[i * k + j] = psi[i * k + j] * a[i]
__global__ void scale_rows_kernel(int rows, int k, const double* __restrict__ psi,
                                  const double* __restrict__ a, double* __restrict__ out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)rows * k) return;
  out[t] = psi[t] * a[t / k];
}

// Column block width N (real columns, multiple of 16, <= 256) of a problem
// with 2k real columns: blocks of at most 128 columns, balanced.  A wider
// block re-reads less of A per output but gives fewer, coarser dependency
// units; 128 keeps a 320-column block in five units.
// Column-block width of the rule: the widest balanced blocks of at most
// 128 real columns (the autotuner may pick up to the accumulator width).
int block_width(int k) {
  const int cols = 2 * k;
  const int nb = (cols + 127) / 128;
  int N = (cols + nb - 1) / nb;
  N = (N + 15) / 16 * 16;
  return std::max(16, std::min(128, N));
}

// Widest column block the accumulator of a split format holds.
int max_block_width(int ns) { return ns == 2 ? KCfg<2>::SLOT : KCfg<3>::SLOT; }

}  // namespace

// ======================================================== host ===========
// Operand slot of one problem: A pieces of its H, B buffers, masters, FP32
// copy of the refinement forcing block.
struct TcSlot {
  int n = 0, kcap = 0, P = 0, pieces = 0;
  const double2* H = nullptr;  // H whose pieces are in A (valid after prepare)
  __nv_bfloat16* A = nullptr;  // MAX_PIECES x n x P
  __nv_bfloat16* B = nullptr;  // 2 buffers x MAX_PIECES x (2 kcap x P)
  float2* M = nullptr;         // 3 x n x kcap
  float2* Rf = nullptr;        // n x kcap
};

// Tiling of a launch: block width N (real columns) and blocks per tile
// group; 0 = the rule (block_width, SMs / row tiles).
struct TcTiling {
  int N = 0, G = 0;
};

struct TcTuned {
  TcTiling t;
  float us = 0.f;
};

struct TcFilterState {
  std::vector<TcSlot> slots;
  std::map<unsigned long long, TcTuned> tuned;  // (n, k / 32, pieces) -> best tiling
  FProb* d_probs = nullptr;
  FSeg* d_segs = nullptr;
  CUtensorMap* d_maps = nullptr;
  int* d_done = nullptr;
  int* d_flags = nullptr;  // [abort, err]
  size_t cap_probs = 0, cap_segs = 0, cap_maps = 0, cap_done = 0;
  bool attr = false;
};

int tc_filter_supported(chfsi_ctx* ctx) { return ctx->cc_major == 10 && ctx->cc_minor == 3; }

static TcFilterState* tc_state(chfsi_ctx* ctx) {
  if (!ctx->tc) ctx->tc = new TcFilterState();
  return ctx->tc;
}

template <typename T>
static void grow(T*& p, size_t& cap, size_t want) {
  if (want <= cap) return;
  cudaFree(p);
  p = nullptr;
  cap = 0;
  CHFSI_CUDA_TRY(cudaMalloc(&p, sizeof(T) * want));
  cap = want;
}

void tc_filter_release(chfsi_ctx* ctx) {
  TcFilterState* s = ctx->tc;
  if (!s) return;
  for (auto& sl : s->slots) {
    cudaFree(sl.A);
    cudaFree(sl.B);
    cudaFree(sl.M);
    cudaFree(sl.Rf);
  }
  cudaFree(s->d_probs);
  cudaFree(s->d_segs);
  cudaFree(s->d_maps);
  cudaFree(s->d_done);
  cudaFree(s->d_flags);
  delete s;
  ctx->tc = nullptr;
}

static TcSlot& tc_slot(chfsi_ctx* ctx, int slot, int n, int k) {
  TcFilterState* s = tc_state(ctx);
  if ((int)s->slots.size() <= slot) s->slots.resize(slot + 1);
  TcSlot& sl = s->slots[slot];
  const int P = (2 * n + 7) / 8 * 8;  // 16-byte row pitch for TMA
  if (sl.n != n || sl.P != P || !sl.A) {
    cudaFree(sl.A);
    sl.A = nullptr;
    sl.H = nullptr;
    sl.pieces = 0;
    CHFSI_CUDA_TRY(cudaMalloc(&sl.A, sizeof(__nv_bfloat16) * MAX_PIECES * (size_t)n * P));
    sl.n = n;
    sl.P = P;
    sl.kcap = 0;
  }
  if (k > sl.kcap) {
    cudaFree(sl.B);
    cudaFree(sl.M);
    cudaFree(sl.Rf);
    sl.B = nullptr;
    sl.M = nullptr;
    sl.Rf = nullptr;
    CHFSI_CUDA_TRY(
        cudaMalloc(&sl.B, sizeof(__nv_bfloat16) * 2 * MAX_PIECES * (size_t)2 * k * P));
    CHFSI_CUDA_TRY(cudaMalloc(&sl.M, sizeof(float2) * 3 * (size_t)n * k));
    CHFSI_CUDA_TRY(cudaMalloc(&sl.Rf, sizeof(float2) * (size_t)n * k));
    sl.kcap = k;
  }
  return sl;
}

void tc_filter_prepare(chfsi_ctx* ctx, int slot, const double2* H, int n, int pieces) {
  TcSlot& sl = tc_slot(ctx, slot, n, 1);
  dim3 grid((2 * n + 255) / 256, n);
  repack_h_kernel<<<grid, 256, 0, ctx->stream>>>(n, sl.P, pieces, H, sl.A, (size_t)n * sl.P);
  chfsi_check_launch("repack_h");
  sl.H = H;
  sl.pieces = pieces;
}

static void launch_with(chfsi_ctx* ctx, int P, const TcBatchItem* items, int ns,
                        const TcTiling& tl) {
  TcFilterState* fs = tc_state(ctx);
  cudaStream_t st = ctx->stream;
  std::vector<FProb> probs(P);
  std::vector<CUtensorMap> maps(9 * (size_t)P);
  int nmax = 16, max_steps = 0;
  for (int p = 0; p < P; ++p) {
    const TcBatchItem& it = items[p];
    const int n = it.n, k = it.k;
    CHFSI_REQUIRE(n >= 1 && k >= 1 && k <= n, "bad filter problem size");
    TcSlot& sl = tc_slot(ctx, it.slot, n, k);
    if (!(it.h_ready && sl.H == it.H && sl.pieces >= ns))
      tc_filter_prepare(ctx, it.slot, it.H, n, ns);
    const size_t a_el = (size_t)n * sl.P, b_el = (size_t)2 * k * sl.P;
    FProb& pr = probs[p];
    pr.n = n;
    pr.k = k;
    pr.P = sl.P;
    pr.kblocks = (2 * n + BK - 1) / BK;
    pr.ntile = tl.N > 0 ? std::min(std::min(tl.N, max_block_width(ns)), (2 * k + 15) / 16 * 16)
                        : block_width(k);
    pr.M = sl.M;
    pr.B = sl.B;
    pr.b_elems = (long long)b_el;
    pr.out = it.out;
    pr.Rf = it.R ? sl.Rf : nullptr;
    nmax = std::max(nmax, pr.ntile);
    for (int q = 0; q < MAX_PIECES; ++q)
      maps[9 * p + q] = make_map(sl.A + (size_t)q * a_el, 2 * n, n, sl.P, BM);
    for (int buf = 0; buf < 2; ++buf)
      for (int q = 0; q < MAX_PIECES; ++q)
        maps[9 * p + 3 + 3 * buf + q] =
            make_map(sl.B + (size_t)(MAX_PIECES * buf + q) * b_el, 2 * n, 2 * k, sl.P, pr.ntile);
    const int* deg = it.deg;
    const int sidx0 = (int)(std::upper_bound(deg, deg + k, 1) - deg);
    const double sigma1 = it.e / (it.lam1 - it.c);
    if (!it.R) {
      // Y_0 -> master 0 and B buffer 0
      split_block_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(
          n, k, sl.P, it.src, 1.0, sl.M, sl.B, b_el, nullptr, 0, nullptr);
    } else {
      // D_1 = a_0 R -> master 1 and B buffer 1; degree-1 columns finished;
      // R in FP32 for the forcing term
      split_block_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(
          n, k, sl.P, it.R, sigma1 / it.e, sl.M + (size_t)n * k,
          sl.B + (size_t)MAX_PIECES * b_el, b_el, it.out, sidx0, sl.Rf);
    }
    chfsi_check_launch("split_block");
    max_steps = std::max(max_steps, deg[k - 1]);
  }
  // Segments in (step, problem) order; tiles block-major within a segment.
  std::vector<FSeg> segs;
  std::vector<int> last_seg(P, -1);
  std::vector<double> sig(P), s1(P);
  for (int p = 0; p < P; ++p) s1[p] = sig[p] = items[p].e / (items[p].lam1 - items[p].c);
  int tiles = 0, counters = 0;
  for (int i = 0; i < max_steps; ++i) {
    for (int p = 0; p < P; ++p) {
      const TcBatchItem& it = items[p];
      const int k = it.k;
      const int* deg = it.deg;
      if (i >= deg[k - 1]) continue;
      if (it.R && i == 0) continue;  // D_1 formed before the launch
      FSeg sg;
      sg.p = p;
      sg.step = i;
      const int s = (int)(std::upper_bound(deg, deg + k, i) - deg);
      sg.s_col = s;
      sg.s_new = (int)(std::upper_bound(deg, deg + k, i + 1) - deg);
      double a, bcoef;
      if (i == 0) {
        a = s1[p] / it.e;
        bcoef = 0.0;
      } else {
        const double sn = 1.0 / (2.0 / s1[p] - sig[p]);
        a = 2.0 * sn / it.e;
        bcoef = -sn * sig[p];
        sig[p] = sn;
      }
      sg.a = (float)a;
      sg.b = (float)bcoef;
      sg.c = (float)it.c;
      sg.cur = i % 3;
      sg.next = (i + 1) % 3;
      sg.prev = (i == 0 || (it.R && i == 1)) ? -1 : (i - 1) % 3;
      sg.bin = i & 1;
      sg.bout = (i + 1) & 1;
      sg.fR = it.R ? it.fR + (size_t)i * k : nullptr;
      const int N = probs[p].ntile;
      sg.mt = (it.n + BM - 1) / BM;
      sg.blk0 = (2 * s) / N;
      sg.nblk = (2 * k + N - 1) / N - sg.blk0;
      // as many blocks per group as keep one group's tiles within the CTAs
      sg.grp = tl.G > 0 ? std::min(tl.G, sg.nblk)
                        : std::max(1, std::min(sg.nblk, ctx->sm_count / sg.mt));
      sg.tile_base = tiles;
      sg.done_base = counters;
      if (last_seg[p] >= 0) {
        const FSeg& d = segs[last_seg[p]];
        sg.dep = last_seg[p];
        sg.dep_blk0 = d.blk0;
        sg.dep_done = d.done_base;
      } else {
        sg.dep = -1;
        sg.dep_blk0 = 0;
        sg.dep_done = 0;
      }
      tiles += sg.mt * sg.nblk;
      counters += sg.nblk;
      last_seg[p] = (int)segs.size();
      segs.push_back(sg);
    }
  }
  if (segs.empty()) return;
  grow(fs->d_probs, fs->cap_probs, (size_t)P);
  grow(fs->d_maps, fs->cap_maps, maps.size());
  grow(fs->d_segs, fs->cap_segs, segs.size());
  grow(fs->d_done, fs->cap_done, (size_t)counters);
  if (!fs->d_flags) CHFSI_CUDA_TRY(cudaMalloc(&fs->d_flags, sizeof(int) * 2));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(fs->d_probs, probs.data(), sizeof(FProb) * P,
                                 cudaMemcpyHostToDevice, st));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(fs->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                 cudaMemcpyHostToDevice, st));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(fs->d_segs, segs.data(), sizeof(FSeg) * segs.size(),
                                 cudaMemcpyHostToDevice, st));
  CHFSI_CUDA_TRY(cudaMemsetAsync(fs->d_done, 0, sizeof(int) * counters, st));
  CHFSI_CUDA_TRY(cudaMemsetAsync(fs->d_flags, 0, sizeof(int) * 2, st));
  const uint32_t stage_bytes = (uint32_t)ns * (BM * BK * 2 + (uint32_t)nmax * BK * 2);
  int stages = (int)((220u * 1024u) / stage_bytes);
  stages = std::max(2, std::min(stages, 6));
  const size_t smem = 1024 + (size_t)stages * stage_bytes + 8 * (2 * stages + 2 * RING + 1) + 64;
  if (!fs->attr) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(tc_filter_kernel<2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(tc_filter_kernel<3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    fs->attr = true;
  }
  void* kfn = ns == 2 ? (void*)tc_filter_kernel<2> : (void*)tc_filter_kernel<3>;
  int per_sm = 0;
  const int threads = ns == 2 ? kthreads<2>() : kthreads<3>();
  CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem));
  if (per_sm < 1) throw ChfsiError{CHFSI_ENOTSUP, "tensor-core filter does not fit on an SM"};
  int grid = std::min(ctx->sm_count * per_sm, tiles);
  const FProb* a0 = fs->d_probs;
  const FSeg* a1 = fs->d_segs;
  int a2 = (int)segs.size();
  int a3 = tiles;
  const CUtensorMap* a4 = fs->d_maps;
  int a5 = nmax;
  int a6 = stages;
  int* a7 = fs->d_done;
  int* a8 = fs->d_flags;
  int* a9 = fs->d_flags + 1;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9};
  double fl = 0.0;
  for (const FSeg& sg : segs)
    fl += 8.0 * (double)items[sg.p].n * items[sg.p].n * (items[sg.p].k - sg.s_col);
  const int slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(threads), args, smem, st));
  chfsi_check_launch("tc_filter");
  kt_end(st, slot, KT_TC, fl, fl * (ns == 2 ? 3.0 : 6.0));
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, fs->d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  if (*h)
    throw ChfsiError{CHFSI_ETIMEOUT, "tensor-core filter: a bounded wait gave up (code " +
                                         std::to_string(*h) + ")"};
}

// Filter launch with a measured tiling (the autotuner, opts.autotune): the
// block width N and the group size decide only which CTA computes which
// output tile; every output element sums the same products in the same K
// order, so all tilings give identical results.  The first single-problem
// launch of each (n, k / 32, pieces) shape times every candidate once (the
// launch is idempotent: it rebuilds its state from Y0 or R), keeps the
// fastest for the context and then runs it; later launches of that shape use
// it directly.  Batched launches use the rule.
void tc_filter_launch(chfsi_ctx* ctx, int P, const TcBatchItem* items, int ns) {
  if (P <= 0) return;
  CHFSI_REQUIRE(ns == 2 || ns == 3, "split pieces must be 2 or 3");
  TcFilterState* fs = tc_state(ctx);
  TcTiling tl;
  if (P == 1 && ctx->opts.autotune) {
    const unsigned long long key = ((unsigned long long)items[0].n << 32) |
                                   ((unsigned long long)((items[0].k + 31) / 32) << 8) |
                                   (unsigned long long)ns;
    auto it = fs->tuned.find(key);
    if (it == fs->tuned.end()) {
      cudaStream_t st = ctx->stream;
      KernelTimer* saved = kt_current();
      kt_install(nullptr);  // the trials are not part of the solve's kernel times
      cudaEvent_t e0, e1;
      CHFSI_CUDA_TRY(cudaEventCreate(&e0));
      CHFSI_CUDA_TRY(cudaEventCreate(&e1));
      TcTuned best;
      best.us = 1e30f;
      try {
        launch_with(ctx, P, items, ns, TcTiling{});  // warm-up (slot buffers, first use)
        for (int N : {64, 96, 128, 160, 192, 224, 256})
          for (int G : {1, 2, 4}) {
            if (N > max_block_width(ns)) continue;
            if (N > (2 * items[0].k + 15) / 16 * 16 + 15) continue;
            TcTiling cand{N, G};
            CHFSI_CUDA_TRY(cudaEventRecord(e0, st));
            launch_with(ctx, P, items, ns, cand);
            CHFSI_CUDA_TRY(cudaEventRecord(e1, st));
            CHFSI_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            CHFSI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (1e3f * ms < best.us) {
              best.us = 1e3f * ms;
              best.t = cand;
            }
          }
      } catch (...) {
        kt_install(saved);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
      }
      kt_install(saved);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      it = fs->tuned.emplace(key, best).first;
    }
    tl = it->second.t;
  }
  launch_with(ctx, P, items, ns, tl);
}

int tc_tuning_table(chfsi_ctx* ctx, int max_entries, int* out) {
  TcFilterState* fs = tc_state(ctx);
  int n = 0;
  for (const auto& kv : fs->tuned) {
    if (n < max_entries && out) {
      int* e = out + 6 * n;
      e[0] = (int)(kv.first >> 32);
      e[1] = (int)((kv.first >> 8) & 0xFFFFFFu) * 32;
      e[2] = (int)(kv.first & 0xFF);
      e[3] = kv.second.t.N;
      e[4] = kv.second.t.G;
      e[5] = (int)kv.second.us;
    }
    ++n;
  }
  return n;
}

// Refinement-form tables for one problem: psi[i][j] = psi_i(lambda_j) and
// the forcing coefficients fR[i][j] = a_i psi_i(lambda_j), (m_k + 1) x k each,
// in context workspaces named after `prefix`.
void tc_defect_tables(chfsi_ctx* ctx, const std::string& prefix, int k, const double* lam,
                      const int* deg_host, double lam1, double c, double e, double** psi_out,
                      double** fR_out) {
  const int mk = deg_host[k - 1];
  std::vector<double> coef(2 * mk + 1, 0.0);
  const double sigma1 = e / (lam1 - c);
  coef[0] = sigma1 / e;
  double sigma = sigma1;
  for (int i = 1; i < mk; ++i) {
    const double sn = 1.0 / (2.0 / sigma1 - sigma);
    coef[2 * i - 1] = 2.0 * sn / e;
    coef[2 * i] = -sn * sigma;
    sigma = sn;
  }
  std::vector<double> ai(mk + 1, 0.0);
  for (int i = 1; i < mk; ++i) ai[i] = coef[2 * i - 1];
  double* dcoef = (double*)ws_get(ctx, (prefix + "tc_coef").c_str(), sizeof(double) * coef.size());
  double* dai = (double*)ws_get(ctx, (prefix + "tc_ai").c_str(), sizeof(double) * (mk + 1));
  double* psi = (double*)ws_get(ctx, (prefix + "tc_psi").c_str(), sizeof(double) * (size_t)(mk + 1) * k);
  double* fR = (double*)ws_get(ctx, (prefix + "tc_fR").c_str(), sizeof(double) * (size_t)(mk + 1) * k);
  double* hbuf = (double*)pinned_get(ctx, sizeof(double) * (coef.size() + ai.size()) + 64);
  std::copy(coef.begin(), coef.end(), hbuf);
  std::copy(ai.begin(), ai.end(), hbuf + coef.size());
  CHFSI_CUDA_TRY(cudaMemcpyAsync(dcoef, hbuf, sizeof(double) * coef.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(dai, hbuf + coef.size(), sizeof(double) * ai.size(),
                                 cudaMemcpyHostToDevice, ctx->stream));
  psi_table_kernel<<<(k + 127) / 128, 128, 0, ctx->stream>>>(k, mk, lam, c, dcoef, psi);
  chfsi_check_launch("psi_table");
  scale_rows_kernel<<<(unsigned)(((size_t)(mk + 1) * k + 255) / 256), 256, 0, ctx->stream>>>(
      mk + 1, k, psi, dai, fR);
  chfsi_check_launch("scale_rows");
  // the host staging buffer is reused by the next call: finish the copies
  CHFSI_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *psi_out = psi;
  *fR_out = fR;
}

void tc_defect_combine(cudaStream_t st, int n, int k, const double2* Y, const int* deg_dev,
                       const double* psi, double2* out) {
  defect_combine_kernel<<<dim3((n + 255) / 256, k), 256, 0, st>>>(n, k, Y, deg_dev, psi, out);
  chfsi_check_launch("defect_combine");
}

// One problem in operand slot 0, H repacked for this call.
void tc_filter_run(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y0,
                   const int* deg_host, double lam1, double c, double e, double2* Yout, int ns) {
  TcBatchItem it{};
  it.H = H;
  it.n = n;
  it.k = k;
  it.src = Y0;
  it.deg = deg_host;
  it.lam1 = lam1;
  it.c = c;
  it.e = e;
  it.out = Yout;
  it.slot = 0;
  it.h_ready = false;
  tc_filter_launch(ctx, 1, &it, ns);
}

// Defect form: Y (degree-sorted), R = HY - Y Lambda (same order), lam (the
// shifts, device, same order), deg_dev (device copy of the degrees).
// Yout = p(H) Y per column.
void tc_filter_run_defect(chfsi_ctx* ctx, const double2* H, int n, int k, const double2* Y,
                          const double2* Rres, const double* lam, const int* deg_host,
                          const int* deg_dev, double lam1, double c, double e, double2* Yout,
                          int ns) {
  double *psi, *fR;
  tc_defect_tables(ctx, "", k, lam, deg_host, lam1, c, e, &psi, &fR);
  TcBatchItem it{};
  it.H = H;
  it.n = n;
  it.k = k;
  it.src = Y;
  it.R = Rres;
  it.fR = fR;
  it.deg = deg_host;
  it.lam1 = lam1;
  it.c = c;
  it.e = e;
  it.out = Yout;
  it.slot = 0;
  it.h_ready = false;
  tc_filter_launch(ctx, 1, &it, ns);
  tc_defect_combine(ctx->stream, n, k, Y, deg_dev, psi, Yout);
}
