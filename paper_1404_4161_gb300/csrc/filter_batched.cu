// Batched persistent split-precision Chebyshev filter: every step of Alg. 2
// for many independent problems of uneven size in ONE cooperative launch.
//
// Work is a list of 128 x N output tiles ordered by (filter step, problem,
// row tile, column tile).  A step of problem p is one "segment"; its tiles
// may only start when every tile of the previous step of p has finished,
// because each output tile reads the whole of Y_i.  CTA b (one per SM, all
// co-resident under the cooperative launch) takes tiles b, b + G, b + 2G,
// ... in increasing order, so every tile a CTA waits for is held by a CTA
// that waits only on earlier steps: the waits always end.  Each wait is
// still bounded (globaltimer) and watches a global abort word, so a fault
// in one CTA turns into CHFSI_ETIMEOUT instead of a hang.
//
// Inside a CTA the roles are those of the single-problem kernel (TMA
// producer, tcgen05.mma issuer, four epilogue warps); the TMEM accumulator
// is handed back and forth with two mbarriers (full / empty), and the
// k-block pipeline keeps its phase across tiles.  An epilogue publishes a
// finished tile with: generic stores -> fence.proxy.async (the next step
// reads them with TMA) -> a per-tile arrival count of the four epilogue
// warps in shared memory (non-blocking) -> the last warp's release add on
// the segment's counter; consumers acquire the counter before their TMA
// or loads.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_ptx.cuh"

using namespace tcx;

namespace {

struct BProb {
  int n, k, P, kblocks, ntile;
  float2* M;           // three FP32 masters, n x k each
  __nv_bfloat16* B;    // [buf0 hi][buf0 lo][buf1 hi][buf1 lo], each 2k x P
  long long b_elems;   // 2k * P
  double2* out;        // FP64 output, n x k
  const double2* R;    // forcing block of the refinement form, or null
};

struct BSeg {
  int p, step, tile_base, mt, nt;
  int s_col, ka, fin_end;
  float a, b, c;
  int cur, prev, next;  // master indices; prev < 0 when b == 0
  int bin, bout;        // B buffers read / written
  int dep, dep_tiles;   // previous segment of the same problem (-1: none)
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

__device__ __forceinline__ int find_seg(const BSeg* segs, int nsegs, int t) {
  int lo = 0, hi = nsegs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Global-memory abort word shared by all CTAs; each CTA also has a local
// copy for its mbarrier waits.
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

__global__ void __launch_bounds__(NTHREADS, 1)
tc_filter_batched_kernel(const BProb* __restrict__ probs, const BSeg* __restrict__ segs, int nsegs,
                         int total_tiles, const CUtensorMap* __restrict__ maps, int nmax,
                         int stages, int* done, int* abort_g_ptr, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t bmax_bytes = (uint32_t)nmax * BK * 2;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * bmax_bytes;
  uint64_t* bars = (uint64_t*)(smem + (size_t)stages * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* accf = bars + 2 * stages;
  uint64_t* acce = accf + 1;
  uint32_t* tmem_slot = (uint32_t*)(acce + 1);
  volatile int* abort_sh = (volatile int*)(tmem_slot + 1);
  int* ep_count = (int*)(tmem_slot + 2);
  volatile int* abort_g = (volatile int*)abort_g_ptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 1);
    *abort_sh = 0;
    *ep_count = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) tmem_alloc(tmem_slot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    uint32_t kbg = 0;
    int issued_lo = 0, issued_hi = 0;  // kbg range of the last stages armed
    for (int t = blockIdx.x; t < total_tiles && !*abort_g; t += gridDim.x) {
      const int si = find_seg(segs, nsegs, t);
      const BSeg& sg = segs[si];
      const BProb& pr = probs[sg.p];
      const int local = t - sg.tile_base;
      const int m0 = (local / sg.nt) * BM;
      const int n0 = (local % sg.nt) * pr.ntile;
      if (sg.dep >= 0 && !wait_count(done + sg.dep, sg.dep_tiles, abort_g, err)) break;
      fence_proxy_async_global();
      const CUtensorMap* mp = maps + (size_t)sg.p * 6;
      const uint32_t bytes = 2 * a_bytes + 2u * (uint32_t)pr.ntile * BK * 2;
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
        tma_load_2d(st, mp + 0, &full[s], kb * BK, m0);
        tma_load_2d(st + a_bytes, mp + 1, &full[s], kb * BK, m0);
        tma_load_2d(st + 2 * a_bytes, mp + 2 + 2 * sg.bin, &full[s], kb * BK,
                    2 * sg.s_col + n0);
        tma_load_2d(st + 2 * a_bytes + bmax_bytes, mp + 3 + 2 * sg.bin, &full[s], kb * BK,
                    2 * sg.s_col + n0);
        issued_hi = (int)kbg + 1;
        issued_lo = issued_hi > stages ? issued_hi - stages : 0;
      }
      if (!ok) break;
    }
    if (*abort_sh || *abort_g) {
      for (int kb = issued_lo; kb < issued_hi; ++kb) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full[kb % stages], (uint32_t)(kb / stages) & 1u) &&
               globaltimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    uint32_t kbg = 0, tcount = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++tcount) {
      const BSeg& sg = segs[find_seg(segs, nsegs, t)];
      const BProb& pr = probs[sg.p];
      if (!wait_bar(acce, (tcount & 1u) ^ 1u, abort_sh, abort_g, err, 6)) break;
      tc_fence_after();
      const uint32_t idesc = idesc_bf16(BM, pr.ntile);
      bool ok = true;
      for (int kb = 0; kb < pr.kblocks; ++kb, ++kbg) {
        const int s = (int)(kbg % (uint32_t)stages);
        const uint32_t ph = (kbg / (uint32_t)stages) & 1u;
        if (!wait_bar(&full[s], ph, abort_sh, abort_g, err, 7)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + (size_t)s * stage_bytes);
        const uint64_t dAh = desc_sw128(sa), dAl = desc_sw128(sa + a_bytes);
        const uint64_t dBh = desc_sw128(sa + 2 * a_bytes);
        const uint64_t dBl = desc_sw128(sa + 2 * a_bytes + bmax_bytes);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t adv = (uint64_t)((kk * 32) >> 4);
          const uint32_t acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
          umma_bf16(tmem, dAh + adv, dBh + adv, idesc, acc0);
          umma_bf16(tmem, dAh + adv, dBl + adv, idesc, 1u);
          umma_bf16(tmem, dAl + adv, dBh + adv, idesc, 1u);
        }
        umma_commit(&empty[s]);
      }
      if (!ok) break;
      umma_commit(accf);
    }
  } else if (warp >= 4) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;
    uint32_t tcount = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++tcount) {
      const int si = find_seg(segs, nsegs, t);
      const BSeg& sg = segs[si];
      const BProb& pr = probs[sg.p];
      const int local = t - sg.tile_base;
      const int m0 = (local / sg.nt) * BM;
      const int n0 = (local % sg.nt) * pr.ntile;
      const bool ok = wait_bar(accf, tcount & 1u, abort_sh, abort_g, err, 8);
      tc_fence_after();
      if (!ok) break;
      if (sg.dep >= 0) (void)ld_acquire(done + sg.dep);  // orders the master reads below
      const int n = pr.n;
      const int row = m0 + q * 32 + lane;
      const size_t coff = (size_t)sg.s_col * n;
      const float2* cur = pr.M + (size_t)sg.cur * n * pr.k + coff;
      const float2* prev = sg.prev >= 0 ? pr.M + (size_t)sg.prev * n * pr.k + coff : nullptr;
      float2* next = pr.M + (size_t)sg.next * n * pr.k + coff;
      const double2* Rs = (sg.fR && pr.R) ? pr.R + coff : nullptr;
      const double* fR = sg.fR ? sg.fR + sg.s_col : nullptr;
      __nv_bfloat16* bh = pr.B + (size_t)(2 * sg.bout) * pr.b_elems + (size_t)(2 * sg.s_col) * pr.P;
      __nv_bfloat16* bl = bh + pr.b_elems;
      double2* out = pr.out + coff;
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
      for (int c0 = 0; c0 < pr.ntile; c0 += 16) {
        float v[16];
        __syncwarp();
        tmem_ld16(tq + (uint32_t)c0, v);
        if (row >= n) continue;
#pragma unroll
        for (int tt = 0; tt < 8; ++tt) {
          const int j = (n0 + c0) / 2 + tt;
          if (j >= sg.ka) break;
          const size_t e = (size_t)row + (size_t)j * n;
          const float2 cu = cur[e];
          float re = sg.a * (v[2 * tt] - sg.c * cu.x);
          float im = sg.a * (v[2 * tt + 1] - sg.c * cu.y);
          if (prev) {
            const float2 pv = prev[e];
            re = fmaf(sg.b, pv.x, re);
            im = fmaf(sg.b, pv.y, im);
          }
          if (Rs) {
            const double f = fR[j];
            const double2 rr = Rs[e];
            re += (float)(f * rr.x);
            im += (float)(f * rr.y);
          }
          next[e] = make_float2(re, im);
          __nv_bfloat16 h, l;
          const size_t r0 = (size_t)(2 * j) * pr.P, r1 = r0 + pr.P;
          split_bf16(re, h, l);
          bh[r0 + row] = h;  bl[r0 + row] = l;
          bh[r1 + n + row] = h;  bl[r1 + n + row] = l;
          split_bf16(im, h, l);
          bh[r1 + row] = h;  bl[r1 + row] = l;
          split_bf16(-im, h, l);
          bh[r0 + n + row] = h;  bl[r0 + n + row] = l;
          if (j < sg.fin_end) out[e] = make_double2((double)re, (double)im);
        }
      }
      // Non-blocking hand-off: the last of the four epilogue warps to finish
      // this tile returns the accumulator to the MMA warp and publishes the
      // tile (no CTA barrier, so an aborting warp cannot block the others).
      tc_fence_before();
      fence_proxy_async_global();
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        const int arrived = atomicAdd(ep_count, 1);
        if (arrived == 4 * (int)tcount + 3) {
          mbar_arrive(acce);
          __threadfence();
          red_release_add(done + si, 1);
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

}  // namespace

// ======================================================== host ===========
struct BatchBufs {
  int n = 0, k = 0, P = 0;
  __nv_bfloat16* A = nullptr;
  __nv_bfloat16* B = nullptr;
  float2* M = nullptr;
};

struct BatchState {
  std::vector<BatchBufs> bufs;
  BProb* d_probs = nullptr;
  BSeg* d_segs = nullptr;
  CUtensorMap* d_maps = nullptr;
  int* d_done = nullptr;
  int* d_flags = nullptr;  // [abort, err]
  size_t cap_probs = 0, cap_segs = 0, cap_maps = 0, cap_done = 0;
  bool attr = false;
};

static BatchState* batch_state(chfsi_ctx* ctx) {
  static thread_local std::unordered_map<chfsi_ctx*, BatchState*> m;
  auto it = m.find(ctx);
  if (it != m.end()) return it->second;
  BatchState* s = new BatchState();
  m[ctx] = s;
  return s;
}

template <typename T>
static void grow(T*& p, size_t& cap, size_t want) {
  if (want <= cap) return;
  cudaFree(p);
  p = nullptr;
  CHFSI_CUDA_TRY(cudaMalloc(&p, sizeof(T) * want));
  cap = want;
}

void tc_filter_batched_release(chfsi_ctx* ctx) {
  BatchState* s = batch_state(ctx);
  for (auto& b : s->bufs) {
    cudaFree(b.A);
    cudaFree(b.B);
    cudaFree(b.M);
  }
  s->bufs.clear();
  cudaFree(s->d_probs);
  cudaFree(s->d_segs);
  cudaFree(s->d_maps);
  cudaFree(s->d_done);
  cudaFree(s->d_flags);
  *s = BatchState();
}

// Column tile per problem: the fewest <= 256-wide tiles, balanced.
int batched_ntile(int k) {
  const int cols = 2 * k;
  const int tiles = (cols + 255) / 256;
  int N = (cols + tiles - 1) / tiles;
  N = (N + 15) / 16 * 16;
  return std::max(32, std::min(256, N));
}

void tc_filter_batched_run(chfsi_ctx* ctx, int P, const TcBatchItem* items) {
  if (P <= 0) return;
  BatchState* bs = batch_state(ctx);
  cudaStream_t st = ctx->stream;
  if ((int)bs->bufs.size() < P) bs->bufs.resize(P);
  std::vector<BProb> probs(P);
  std::vector<CUtensorMap> maps(6 * (size_t)P);
  std::vector<BSeg> segs;
  int nmax = 32, max_steps = 0;
  for (int p = 0; p < P; ++p) {
    const TcBatchItem& it = items[p];
    const int n = it.n, k = it.k;
    CHFSI_REQUIRE(n >= 1 && k >= 1 && k <= n, "bad batched problem size");
    BatchBufs& b = bs->bufs[p];
    const int Pp = (2 * n + 7) / 8 * 8;
    if (b.n != n || b.k < k || b.P != Pp) {
      cudaFree(b.A);
      cudaFree(b.B);
      cudaFree(b.M);
      b = BatchBufs();
      CHFSI_CUDA_TRY(cudaMalloc(&b.A, sizeof(__nv_bfloat16) * 2 * (size_t)n * Pp));
      CHFSI_CUDA_TRY(cudaMalloc(&b.B, sizeof(__nv_bfloat16) * 4 * (size_t)2 * k * Pp));
      CHFSI_CUDA_TRY(cudaMalloc(&b.M, sizeof(float2) * 3 * (size_t)n * k));
      b.n = n;
      b.k = k;
      b.P = Pp;
    }
    const size_t a_el = (size_t)n * Pp, b_el = (size_t)2 * k * Pp;
    tc_repack_h(st, n, Pp, it.H, b.A, b.A + a_el);
    BProb& pr = probs[p];
    pr.n = n;
    pr.k = k;
    pr.P = Pp;
    pr.kblocks = (2 * n + BK - 1) / BK;
    pr.ntile = batched_ntile(k);
    pr.M = b.M;
    pr.B = b.B;
    pr.b_elems = (long long)b_el;
    pr.out = it.out;
    pr.R = it.R;
    nmax = std::max(nmax, pr.ntile);
    maps[6 * p + 0] = make_map(b.A, 2 * n, n, Pp, BM);
    maps[6 * p + 1] = make_map(b.A + a_el, 2 * n, n, Pp, BM);
    for (int buf = 0; buf < 2; ++buf) {
      maps[6 * p + 2 + 2 * buf] = make_map(b.B + (size_t)(2 * buf) * b_el, 2 * n, 2 * k, Pp,
                                           pr.ntile);
      maps[6 * p + 3 + 2 * buf] = make_map(b.B + (size_t)(2 * buf + 1) * b_el, 2 * n, 2 * k,
                                           Pp, pr.ntile);
    }
    const int* deg = it.deg;
    const int sidx0 = (int)(std::upper_bound(deg, deg + k, 1) - deg);
    const double sigma1 = it.e / (it.lam1 - it.c);
    if (!it.R) {
      // Y_0 -> master 0 and B buffer 0
      tc_split_block(st, n, k, Pp, it.src, 1.0, b.M, b.B, b.B + b_el, nullptr, 0);
    } else {
      // D_1 = a_0 R -> master 1 and B buffer 1; degree-1 columns finished
      tc_split_block(st, n, k, Pp, it.R, sigma1 / it.e, b.M + (size_t)n * k,
                     b.B + 2 * b_el, b.B + 3 * b_el, it.out, sidx0);
    }
    max_steps = std::max(max_steps, deg[k - 1]);
  }
  // Segments in (step, problem) order.
  std::vector<int> last_seg(P, -1), last_tiles(P, 0);
  std::vector<double> sig(P), s1(P);
  for (int p = 0; p < P; ++p) s1[p] = sig[p] = items[p].e / (items[p].lam1 - items[p].c);
  int tiles = 0;
  for (int i = 0; i < max_steps; ++i) {
    for (int p = 0; p < P; ++p) {
      const TcBatchItem& it = items[p];
      const int k = it.k;
      const int* deg = it.deg;
      if (i >= deg[k - 1]) continue;
      if (it.R && i == 0) continue;  // D_1 formed before the launch
      BSeg sg;
      sg.p = p;
      sg.step = i;
      const int s = (int)(std::upper_bound(deg, deg + k, i) - deg);
      const int s_new = (int)(std::upper_bound(deg, deg + k, i + 1) - deg);
      sg.s_col = s;
      sg.ka = k - s;
      sg.fin_end = s_new - s;
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
      sg.mt = (it.n + BM - 1) / BM;
      sg.nt = (2 * sg.ka + probs[p].ntile - 1) / probs[p].ntile;
      sg.tile_base = tiles;
      sg.dep = last_seg[p];
      sg.dep_tiles = last_tiles[p];
      tiles += sg.mt * sg.nt;
      last_seg[p] = (int)segs.size();
      last_tiles[p] = sg.mt * sg.nt;
      segs.push_back(sg);
    }
  }
  if (segs.empty()) return;
  grow(bs->d_probs, bs->cap_probs, (size_t)P);
  grow(bs->d_maps, bs->cap_maps, maps.size());
  grow(bs->d_segs, bs->cap_segs, segs.size());
  grow(bs->d_done, bs->cap_done, segs.size());
  if (!bs->d_flags) CHFSI_CUDA_TRY(cudaMalloc(&bs->d_flags, sizeof(int) * 2));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(bs->d_probs, probs.data(), sizeof(BProb) * P,
                                 cudaMemcpyHostToDevice, st));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(bs->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                                 cudaMemcpyHostToDevice, st));
  CHFSI_CUDA_TRY(cudaMemcpyAsync(bs->d_segs, segs.data(), sizeof(BSeg) * segs.size(),
                                 cudaMemcpyHostToDevice, st));
  CHFSI_CUDA_TRY(cudaMemsetAsync(bs->d_done, 0, sizeof(int) * segs.size(), st));
  CHFSI_CUDA_TRY(cudaMemsetAsync(bs->d_flags, 0, sizeof(int) * 2, st));
  const uint32_t stage_bytes = 2u * BM * BK * 2 + 2u * (uint32_t)nmax * BK * 2;
  int stages = (int)((220u * 1024u) / stage_bytes);
  stages = std::max(2, std::min(stages, 6));
  const size_t smem = 1024 + (size_t)stages * stage_bytes + 8 * (2 * stages + 2) + 32;
  if (!bs->attr) {
    CHFSI_CUDA_TRY(cudaFuncSetAttribute(tc_filter_batched_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    bs->attr = true;
  }
  int per_sm = 0;
  CHFSI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_filter_batched_kernel,
                                                               NTHREADS, smem));
  if (per_sm < 1) throw ChfsiError{CHFSI_ENOTSUP, "batched filter does not fit on an SM"};
  int grid = std::min(ctx->sm_count * per_sm, tiles);
  const BProb* a0 = bs->d_probs;
  const BSeg* a1 = bs->d_segs;
  int a2 = (int)segs.size();
  int a3 = tiles;
  const CUtensorMap* a4 = bs->d_maps;
  int a5 = nmax;
  int a6 = stages;
  int* a7 = bs->d_done;
  int* a8 = bs->d_flags;
  int* a9 = bs->d_flags + 1;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9};
  const int slot = kt_begin(st);
  CHFSI_CUDA_TRY(cudaLaunchCooperativeKernel((void*)tc_filter_batched_kernel, dim3(grid),
                                             dim3(NTHREADS), args, smem, st));
  chfsi_check_launch("tc_filter_batched");
  double fl = 0.0;
  for (const BSeg& sg : segs) fl += 8.0 * (double)items[sg.p].n * items[sg.p].n * sg.ka;
  kt_end(st, slot, KT_TC, fl);
  int* h = (int*)pinned_get(ctx, 64);
  CHFSI_CUDA_TRY(cudaMemcpyAsync(h, bs->d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHFSI_CUDA_TRY(cudaStreamSynchronize(st));
  if (*h)
    throw ChfsiError{CHFSI_ETIMEOUT, "batched filter: a bounded wait gave up (code " +
                                         std::to_string(*h) + ")"};
}
