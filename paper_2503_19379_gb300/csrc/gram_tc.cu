// Complex64 Gram products on the tensor cores (tcgen05, TF32 operands with a three-term split).
//
// A complex inner product over interleaved (re, im) pairs is two real inner products over the 2L floats:
//   Re a^H b = sum_l (a_re b_re + a_im b_im) = <a, b>,     Im a^H b = sum_l (a_re b_im - a_im b_re) = <a~, b>,
// where a~ replaces every pair (re, im) of a by (-im, re). For a panel A (p columns) and a panel B1 (q columns)
// one real product
//   D = [A; A~] [B]^T        M = 128 rows (2p used), N = q (or q + p), K = 2L
// gives Re A^H B (rows < p) and Im A^H B (rows p .. 2p-1). The Gram pair of the Rayleigh-Ritz step
// (G = S^H S, H = S^H (Op S), the projected pencil of the block search space) is the case A = S, B = [Op S; S].
//
// Precision: every FP32 value x is split x = hi + lo, hi = tf32(x), lo = tf32(x - hi) (round to nearest), and the
// product is formed as hi.hi + (hi.lo + lo.hi); the neglected lo.lo term and the rounding of lo are ~2^-22 relative.
// The tensor core's FP32 accumulator does not round to nearest on every addition (its error grows with the number
// of additions into one accumulator), so hi.hi goes to TMEM accumulators that are drained every TC_GROUP K tiles
// into FP32 registers (round-to-nearest CUDA-core additions) and restarted; two hi.hi accumulators alternate so
// that the MMAs run on while one is drained. Every drained group holds at most 4 TC_GROUP additions of hi.hi,
// which keeps the result at the accuracy of an FP32 CUDA-core product. The two cross terms, ~2^-11 of hi.hi, go to
// a third accumulator that is drained once at the end of the chunk: its accumulation error is 2^-11 times that of
// an undrained hi.hi accumulator, far below FP32 rounding. Three accumulators of N columns fit TMEM's 512 columns
// for N <= 160, which takes the mixed solve's coupled pencil at 19 block columns (N = 2 * 64 + 32).
//
// Structure (one CTA per (k-point, K-chunk), 20 warps):
//   warp 0       one thread issues 2D tensor-map copies (cp.async.bulk.tensor, 128-byte swizzle) of the A and B1
//                tiles (32 floats x rows) into a staging ring of up to 4 stages of 2 K tiles each;
//   warp 1       one thread issues the tcgen05.mma chain (12 per 32-float K tile) into the TMEM accumulators;
//   warps 2..7   turn each staged tile into the hi/lo operand tiles of the K-major layout the tensor core reads
//                (rows of 128 bytes, 16-byte chunks XOR-ed with the row index mod 8, as the copy left them; every
//                block of rows starts at a multiple of 8, so a chunk keeps its position), double buffered against
//                the MMAs;
//   warps 8..19  drain the accumulators (tcgen05.ld: TMEM lane quarter = warp % 4, three warps per quarter
//                splitting the columns in 32-column chunks) into registers and finally write FP64 partial sums per
//                chunk, which the Gram reduction kernels add up.
// Every wait is bounded in time: a wait that runs out raises an abort flag that the other roles observe, copies and
// MMAs in flight are drained (again with a bound), TMEM is released and an error flag is left for the host.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "pc_internal.cuh"

namespace pc {

namespace {

constexpr int TC_THREADS = 640;
constexpr int TC_KT = 32;     // floats of K per tile (one 128-byte swizzle row)
constexpr int TC_SPT = 2;     // K tiles per staging stage: each row arrives as a 256-byte run
constexpr int TC_M = 128;     // MMA rows
constexpr int TC_GROUP = 2;   // K tiles per accumulator drain
constexpr int TC_NTR = 6;     // transform warps (2..7)
constexpr int TC_NDR = 12;    // drain warps (8..19), three per TMEM lane quarter
constexpr int TC_NMAX = 160;  // MMA columns: three accumulators of N columns in the 512 TMEM columns
constexpr int TC_MAXT = 512;  // K tiles per chunk at most: the drain's FP32 running sums span <= 256 groups
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;  // 1 s: a kernel call takes milliseconds

__device__ int g_gram_tc_error = 0;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the completion of the phase of the given parity. Returns false when the abort flag is (or gets) set,
// or after TC_WAIT_NS, in which case it sets the flag. With honour_abort = false only the time bound ends the wait
// (used to drain operations in flight).
__device__ bool bar_wait(uint32_t bar, uint32_t parity, volatile int *abort, bool honour_abort = true) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (bar_try_wait(bar, parity)) return true;
    if ((it & 15) == 15) {
      if (honour_abort && *abort) return false;
      const unsigned long long t = gtimer();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > TC_WAIT_NS) {
        *abort = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// 16 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
}
// adds 32 accumulator columns (two 16-column loads) into acc
__device__ __forceinline__ void tmem_add32(uint32_t taddr, float (&acc)[32]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    uint32_t r[16];
    tmem_ld16(taddr + (uint32_t)(16 * s), r);
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[16 * s + k] += __uint_as_float(r[k]);
  }
}

struct TcArgs {
  long cppA, cppB;      // columns per k-point panel (panel strides / L): tensor-map row of (b, c) = b * cpp + c
  long L;
  int p, q;             // columns of A and of B1
  int PB, QB;           // padded row counts (multiples of 8); the B operand is rows [0, N) of the operand region
  int RB, q2;           // pair mode with a coupling block: B1 = [B1a (QB - RB rows); R (RB rows, q2 used)], the
                        // second part from its own tensor (RB = 0: none)
  long cppR;            // columns per k-point panel of R
  int N;                // MMA N: QB + PB when pair (B = [B1; A]), else QB (multiple of 16, <= TC_NMAX)
  int pair;             // pair: outputs G = A^H A and H = A^H B1 (upper triangles); else A^H B1 (p x q)
  int transpose;        // general mode: write the conjugate transpose (B1^H A, q x p) instead
  int ns;               // staging stages
  int ktiles, tpc, nchunk;
  int nc;                // accumulator columns (N rounded up to 32): hi.hi sets at 0 and nc, cross terms at 2 nc
  uint32_t tmem_cols;    // allocated TMEM columns (3 nc rounded up to a power of two)
  uint32_t idesc;
  double *partG, *partH;  // pair: [nb][nchunk][p][p] double2 each; general: partH = [nb][nchunk][p][q]
  double *partQ;          // coupling block (RB > 0): R^H A as [nb][nchunk][q2][p] double2
  const int *act;
};

__global__ void __launch_bounds__(TC_THREADS, 1) gram_tc_kernel(const TcArgs a, const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB,
                                                                const __grid_constant__ CUtensorMap tmR) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *const sm = smem_raw + (base - raw);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ns = a.ns;
  const uint32_t region = (uint32_t)(a.QB + TC_M) * 128u;  // bytes of one hi (or lo) operand region
  const uint32_t opbuf = 2u * region;                       // hi + lo
  const uint32_t tile_bytes = (uint32_t)(a.PB + a.QB) * 128u;  // one staged K tile: A rows, then B1 rows
  const uint32_t stage_bytes = TC_SPT * tile_bytes;
  const uint32_t off_stage = 2u * opbuf;
  const uint32_t off_bar = off_stage + (uint32_t)ns * stage_bytes;
  // barriers: full[ns], empty[ns], opready[2], opfree[2], accfull[2], accempty[2], done
  const uint32_t bar_full = base + off_bar, bar_empty = bar_full + 8u * ns, bar_ready = bar_empty + 8u * ns,
                 bar_free = bar_ready + 16u, bar_afull = bar_free + 16u, bar_aempty = bar_afull + 16u,
                 bar_done = bar_aempty + 16u;
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(sm + off_bar + 8u * (2 * ns + 9));
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_holder + 1);

  const int bi = blockIdx.y, chunk = blockIdx.x;
  const int b = a.act ? a.act[bi] : bi;
  const int t_begin = chunk * a.tpc;
  const int ntile = min(a.ktiles, t_begin + a.tpc) - t_begin;  // >= 1 by construction of the chunking
  const int ngroup = (ntile + TC_GROUP - 1) / TC_GROUP;

  // zero the operand buffers and the staging ring (rows past p / q stay zero), then make those writes visible
  // to the async proxy (tensor core, bulk copies)
  {
    float4 *z = reinterpret_cast<float4 *>(sm);
    const int nz = (int)(off_bar / 16u);
    for (int i = threadIdx.x; i < nz; i += TC_THREADS) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    fence_proxy_async();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      bar_init(bar_full + 8u * s, 1);
      bar_init(bar_empty + 8u * s, TC_NTR);
    }
    for (int u = 0; u < 2; ++u) {
      bar_init(bar_ready + 8u * u, TC_NTR);
      bar_init(bar_free + 8u * u, 1);
      bar_init(bar_afull + 8u * u, 1);
      bar_init(bar_aempty + 8u * u, TC_NDR);
    }
    bar_init(bar_done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_holder)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ------------------------------------------------ producer
    // whole boxes, TC_SPT tiles per stage (rows or tiles past the tensor are zero-filled; a last stage's second tile
    // past the chunk is loaded and not used)
    const uint32_t tx = stage_bytes;
    const int yA = (int)(b * a.cppA), yB = (int)(b * a.cppB), yR = (int)(b * a.cppR);
    const int nstage = (ntile + TC_SPT - 1) / TC_SPT;
    int issued = 0;
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      if (a.RB > 0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmR)) : "memory");
      for (int q = 0; q < nstage; ++q) {
        const int s = q % ns;
        if (!bar_wait(bar_empty + 8u * s, ((q / ns) & 1) ^ 1, abort)) break;
        bar_expect_tx(bar_full + 8u * s, tx);
        const uint32_t st = base + off_stage + (uint32_t)s * stage_bytes;
#pragma unroll
        for (int h = 0; h < TC_SPT; ++h) {
          const int x = (t_begin + q * TC_SPT + h) * TC_KT;  // float offset: a multiple of 32 (128 bytes)
          tma_load_2d(st + h * tile_bytes, &tmA, x, yA, bar_full + 8u * s);
          tma_load_2d(st + h * tile_bytes + (uint32_t)a.PB * 128u, &tmB, x, yB, bar_full + 8u * s);
          if (a.RB > 0)
            tma_load_2d(st + h * tile_bytes + (uint32_t)(a.PB + a.QB - a.RB) * 128u, &tmR, x, yR, bar_full + 8u * s);
        }
        issued = q + 1;
      }
      // drain: the last use of every stage must have landed before the CTA may exit
      for (int q = max(0, issued - ns); q < issued; ++q)
        bar_wait(bar_full + 8u * (q % ns), (q / ns) & 1, abort, false);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      for (int g = 0; g < ngroup && ok; ++g) {
        const int v = g & 1;
        if (!bar_wait(bar_aempty + 8u * v, ((g >> 1) & 1) ^ 1, abort)) break;
        const uint32_t dA = tmem + (uint32_t)(v * a.nc), dX = tmem + (uint32_t)(2 * a.nc);
        const int t1 = min(ntile, (g + 1) * TC_GROUP);
        for (int t = g * TC_GROUP; t < t1; ++t) {
          const int u = t & 1;
          if (!bar_wait(bar_ready + 8u * u, (t >> 1) & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t hi = base + (uint32_t)u * opbuf, lo = hi + region;
          const uint32_t aoff = (uint32_t)a.QB * 128u;
          const bool first = t == g * TC_GROUP;
#pragma unroll
          for (int ks = 0; ks < TC_KT / 8; ++ks) {
            const uint32_t ko = (uint32_t)ks * 32u;
            const uint64_t ahi = sdesc(hi + aoff + ko), alo = sdesc(lo + aoff + ko);
            const uint64_t bhi = sdesc(hi + ko), blo = sdesc(lo + ko);
            const uint32_t acc = (first && ks == 0) ? 0u : 1u;
            const uint32_t accx = (t == 0 && ks == 0) ? 0u : 1u;  // cross terms: the whole chunk in one accumulator
            mma_tf32(dA, ahi, bhi, a.idesc, acc);
            mma_tf32(dX, ahi, blo, a.idesc, accx);
            mma_tf32(dX, alo, bhi, a.idesc, 1u);
          }
          mma_commit(bar_free + 8u * u);
        }
        if (ok) mma_commit(bar_afull + 8u * v);
      }
      // everything issued has completed once `done` fires; on abort wait for that here (bounded)
      mma_commit(bar_done);
      if (*abort) bar_wait(bar_done, 0, abort, false);
    }
    __syncwarp();
  } else if (warp < 2 + TC_NTR) {
    // ------------------------------------------------ operand transform
    const int tt = threadIdx.x - 64;
    const int nel = (a.PB + a.QB) * 8;  // 16-byte chunks per staged tile
    for (int t = 0; t < ntile; ++t) {
      const int q = t / TC_SPT, hsub = t - q * TC_SPT;
      const int s = q % ns, u = t & 1;
      if (!bar_wait(bar_full + 8u * s, (q / ns) & 1, abort)) break;
      if (!bar_wait(bar_free + 8u * u, ((t >> 1) & 1) ^ 1, abort)) break;
      const unsigned char *st = sm + off_stage + (size_t)s * stage_bytes + (size_t)hsub * tile_bytes;
      unsigned char *hi = sm + (size_t)u * opbuf, *lo = hi + region;
      for (int e = tt; e < nel; e += 32 * TC_NTR) {
        const int row = e >> 3, pc = e & 7;  // physical 16-byte chunk, kept in every row it is copied to
        const float4 v = *reinterpret_cast<const float4 *>(st + row * 128 + pc * 16);
        float4 h, l;
        h.x = tf32_rna(v.x);
        h.y = tf32_rna(v.y);
        h.z = tf32_rna(v.z);
        h.w = tf32_rna(v.w);
        l.x = tf32_rna(v.x - h.x);
        l.y = tf32_rna(v.y - h.y);
        l.z = tf32_rna(v.z - h.z);
        l.w = tf32_rna(v.w - h.w);
        int R;
        if (row < a.PB) {
          // A row: at QB + row, and its (-im, re) partner at QB + PB + row
          R = a.QB + row;
          const int R2 = R + a.PB;
          const uint32_t o2 = (uint32_t)R2 * 128u + (uint32_t)pc * 16u;
          *reinterpret_cast<float4 *>(hi + o2) = make_float4(-h.y, h.x, -h.w, h.z);
          *reinterpret_cast<float4 *>(lo + o2) = make_float4(-l.y, l.x, -l.w, l.z);
        } else {
          R = row - a.PB;  // B1 row
        }
        const uint32_t o = (uint32_t)R * 128u + (uint32_t)pc * 16u;
        *reinterpret_cast<float4 *>(hi + o) = h;
        *reinterpret_cast<float4 *>(lo + o) = l;
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        if (hsub == TC_SPT - 1 || t == ntile - 1) bar_arrive(bar_empty + 8u * s);  // stage consumed
        bar_arrive(bar_ready + 8u * u);
      }
    }
  } else {
    // ------------------------------------------------ accumulator drain and epilogue
    const int dw = warp - (2 + TC_NTR);  // 0..11
    const int qd = warp & 3;            // TMEM lane quarter
    const int slot = dw >> 2;           // column chunks slot, slot + 3 (32 columns each)
    float acc[2][32];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[h][k] = 0.f;
    const uint32_t lanebase = (uint32_t)(qd * 32) << 16;
    bool ok = true;
    for (int g = 0; g < ngroup; ++g) {
      const int v = g & 1;
      if (!bar_wait(bar_afull + 8u * v, (g >> 1) & 1, abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t dA = tmem + lanebase + (uint32_t)(v * a.nc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c0 = (slot + 3 * h) * 32;
        if (c0 < a.N) tmem_add32(dA + (uint32_t)c0, acc[h]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(bar_aempty + 8u * v);
    }
    // the cross terms, once every MMA of the chunk has completed
    if (ok && bar_wait(bar_done, 0, abort)) {
      tc_fence_after();
      const uint32_t dX = tmem + lanebase + (uint32_t)(2 * a.nc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c0 = (slot + 3 * h) * 32;
        if (c0 < a.N) tmem_add32(dX + (uint32_t)c0, acc[h]);
      }
    } else {
      ok = false;
    }
    if (__all_sync(0xffffffffu, ok)) {
      const int i = qd * 32 + lane;  // accumulator row
      const bool im = i >= a.PB;
      const int ii = im ? i - a.PB : i;
      if (i < 2 * a.PB && ii < a.p) {
        const long oG = ((long)bi * a.nchunk + chunk) * a.p * (a.pair ? a.p : a.q);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c0 = (slot + 3 * h) * 32;
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int j = c0 + k;
            const double val = (double)acc[h][k];
            if (a.pair) {
              const int QA = a.QB - a.RB;  // rows of B1a
              if (j >= QA && j < a.QB) {
                // coupling block: (A^H R)_{ii, jq}, stored conjugate-transposed as (R^H A)_{jq, ii}
                const int jq = j - QA;
                if (jq < a.q2) {
                  const long oQ = ((long)bi * a.nchunk + chunk) * a.q2 * a.p;
                  a.partQ[2 * (oQ + (long)jq * a.p + ii) + im] = im ? -val : val;
                }
                continue;
              }
              const bool isH = j < a.QB;
              const int jj = isH ? j : j - a.QB;
              if (j < a.N && jj < a.p && ii <= jj)
                (isH ? a.partH : a.partG)[2 * (oG + (long)ii * a.p + jj) + im] = val;
            } else if (j < a.q) {
              if (a.transpose)
                a.partH[2 * (oG + (long)j * a.p + ii) + im] = im ? -val : val;
              else
                a.partH[2 * (oG + (long)ii * a.q + j) + im] = val;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
  if (threadIdx.x == 0 && *abort) atomicExch(&g_gram_tc_error, 1);
}

constexpr int TC_SMEM_MAX = 232448;  // opt-in shared memory per block

size_t tc_smem(int PB, int QB, int ns) {
  return 1024 + 4 * (size_t)(QB + TC_M) * 128 + (size_t)ns * TC_SPT * (PB + QB) * 128 + 8 * (2 * ns + 9) + 16;
}

// chunks per k-point: at least ktiles / TC_MAXT (the drain adds each chunk's K tiles in FP32 registers, whose
// rounding grows with the number of additions: a chunk of thousands of tiles, as a large batch with few chunks per
// k-point would have, leaves errors of several 1e-6 relative in the Gram entries, enough to stall LOBPCG near a
// relative residual of 1e-6), and whole waves of one CTA per SM where possible, within the partial-sum scratch
int tc_chunks(int nb, int ktiles, long maxc) {
  const int nsm = sm_count();
  const long cmin = std::min<long>((ktiles + TC_MAXT - 1) / TC_MAXT, maxc);
  int best = 1;
  double beff = 0.0;
  for (int w = 1; w <= 64; ++w) {
    long c = std::max<long>(cmin, (long)w * nsm / nb);
    c = std::max<long>(1, std::min<long>({c, (long)ktiles, maxc}));
    const long ctas = (long)nb * c;
    const double eff = (double)ctas / ((double)nsm * ((ctas + nsm - 1) / nsm));
    if (eff > beff + 0.02) {
      beff = eff;
      best = (int)c;
    }
  }
  return std::max(1, best);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// rows of a panel array as a 2D FP32 tensor: x = float offset along a column (2L), y = b * cpp + column
bool make_map(CUtensorMap *map, const void *base, long L, long rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * L), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(8 * L)};
  const cuuint32_t box[2] = {(cuuint32_t)TC_KT, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// pair mode with R (q2 > 0): B1 = [B; R], the coupling block R^H A written to partQ (after the G and H partials)
int launch_tc(int nb, int nb_alloc, long L, int p, int q, bool pair, const void *A, long sa, const void *B, long sb,
              double2 *part, size_t scratch_bytes, cudaStream_t st, const int *act, int *nchunk_out,
              bool transpose = false, const void *R = nullptr, long sr = 0, int q2 = 0) {
  TcArgs a{};
  a.cppA = sa / L;
  a.cppB = sb / L;
  a.cppR = q2 > 0 ? sr / L : 0;
  a.L = L;
  a.p = p;
  a.q = q;
  a.q2 = pair ? q2 : 0;
  a.PB = (p + 7) / 8 * 8;
  a.RB = a.q2 > 0 ? (a.q2 + 7) / 8 * 8 : 0;
  if (a.RB > 0 && (2 * a.PB + a.RB) % 16 != 0) a.RB += 8;  // the MMA's N must be a multiple of 16
  a.QB = pair ? a.PB + a.RB : (q + 15) / 16 * 16;
  a.N = pair ? a.QB + a.PB : a.QB;
  if (a.N > TC_NMAX) return PC_EUNSUPPORTED;
  a.pair = pair ? 1 : 0;
  a.transpose = transpose ? 1 : 0;
  a.ktiles = (int)(2 * L / TC_KT);
  int ns = 4;
  while (ns > 2 && tc_smem(a.PB, a.QB, ns) > (size_t)TC_SMEM_MAX) --ns;
  if (tc_smem(a.PB, a.QB, ns) > (size_t)TC_SMEM_MAX) return PC_EUNSUPPORTED;
  a.ns = ns;
  const size_t per_chunk = sizeof(double2) * (size_t)nb * p * (pair ? 2 * p + a.q2 : q);
  const long maxc = (long)std::min<size_t>(scratch_bytes / per_chunk, 4096);
  if (maxc < 1) return PC_EUNSUPPORTED;
  int c = tc_chunks(nb, a.ktiles, maxc);
  a.tpc = (a.ktiles + c - 1) / c;
  c = (a.ktiles + a.tpc - 1) / a.tpc;
  a.nchunk = c;
  // instruction descriptor: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major,
  // N >> 3 at bits 17-22, M >> 4 at bits 24-28
  a.idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(a.N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
  a.nc = (a.N + 31) / 32 * 32;
  a.tmem_cols = 32;
  while (a.tmem_cols < (uint32_t)(3 * a.nc)) a.tmem_cols *= 2;
  a.partG = reinterpret_cast<double *>(part);
  a.partH = pair ? reinterpret_cast<double *>(part + (size_t)nb * c * p * p) : reinterpret_cast<double *>(part);
  a.partQ = a.q2 > 0 ? reinterpret_cast<double *>(part + 2 * (size_t)nb * c * p * p) : nullptr;
  a.act = act;
  static bool configured = false;
  if (!configured) {
    PC_CK(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX));
    configured = true;
  }
  // a CTA that takes all 512 TMEM columns must have its SM to itself: ask for more than half the shared memory
  size_t smem = tc_smem(a.PB, a.QB, ns);
  if (a.tmem_cols == 512) smem = std::max<size_t>(smem, TC_SMEM_MAX / 2 + 4096);
  CUtensorMap tmA, tmB, tmR;
  const int brows = a.QB - a.RB;  // rows of the B tile
  if (!make_map(&tmA, A, L, (long)(nb_alloc - 1) * a.cppA + p, a.PB) ||
      !make_map(&tmB, B, L, (long)(nb_alloc - 1) * a.cppB + q, brows))
    return PC_EUNSUPPORTED;
  if (a.RB > 0) {
    if (!make_map(&tmR, R, L, (long)(nb_alloc - 1) * a.cppR + a.q2, a.RB)) return PC_EUNSUPPORTED;
  } else {
    tmR = tmB;  // not read
  }
  gram_tc_kernel<<<dim3(c, nb), TC_THREADS, smem, st>>>(a, tmA, tmB, tmR);
  PC_CK_LAUNCH();
  *nchunk_out = c;
  return PC_OK;
}

bool tc_enabled() {
  static int on = -1;
  if (on < 0) {
    const char *e = getenv("PC_GRAM_TC");
    on = (e && e[0] == '0') ? 0 : 1;
  }
  return on == 1;
}

bool tc_shape_ok(long L, int p, int q, const void *A, long sa, const void *B, long sb) {
  if (!tc_enabled()) return false;
  if (L <= 0 || L % (TC_KT / 2) != 0) return false;  // whole 32-float tiles
  if (p < 1 || p > 64 || q < 1 || q > 128) return false;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return false;
  if (sa % L != 0 || sb % L != 0) return false;  // panels of whole columns: one 2D tensor per panel array
  return encode_fn() != nullptr;
}

}  // namespace

// chunks per k-point that the tensor-core Gram takes at least, for panels of L rows (partial-sum scratch sizing)
int tc_min_chunks(long L) { return (int)((2 * L / TC_KT + TC_MAXT - 1) / TC_MAXT); }

// G = S^H S and H = S^H AS (complex64 panels, p <= 64) on the tensor cores; PC_EUNSUPPORTED when the shape or
// alignment does not fit (the caller then takes the CUDA-core kernel).
int launch_gram_pair_tc(int nb, long L, int p, const void *S, const void *AS, long ss, void *G, void *H,
                        void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc, long sg) {
  if (!tc_shape_ok(L, p, p, S, ss, AS, ss)) return PC_EUNSUPPORTED;
  int c = 0;
  double2 *part = static_cast<double2 *>(scratch);
  int rc = launch_tc(nb, nb_alloc > 0 ? nb_alloc : nb, L, p, p, true, S, ss, AS, ss, part, scratch_bytes, st, act,
                     &c);
  if (rc) return rc;
  launch_gram_pair_reduce(nb, c, p, part, act, G, H, st, sg);
  PC_CK_LAUNCH();
  return PC_OK;
}

// G = S^H S, H = S^H AS and RQ = R^H S (q2 x p, row stride p) in one pass over [S | AS | R] (complex64, 2 p + q2
// rounded up <= 160 MMA columns); PC_EUNSUPPORTED as above.
int launch_gram_pair_coupled_tc(int nb, long L, int p, int q2, const void *S, const void *AS, long ss, const void *R,
                                long sr, void *G, void *H, void *RQ, void *scratch, size_t scratch_bytes,
                                cudaStream_t st, const int *act, int nb_alloc, long sg, long srq) {
  if (q2 < 1 || !tc_shape_ok(L, p, p, S, ss, AS, ss) || !tc_shape_ok(L, q2, q2, R, sr, R, sr))
    return PC_EUNSUPPORTED;
  int c = 0;
  double2 *part = static_cast<double2 *>(scratch);
  int rc = launch_tc(nb, nb_alloc > 0 ? nb_alloc : nb, L, p, p, true, S, ss, AS, ss, part, scratch_bytes, st, act,
                     &c, false, R, sr, q2);
  if (rc) return rc;
  launch_gram_pair_reduce(nb, c, p, part, act, G, H, st, sg);
  PC_CK_LAUNCH();
  launch_gram_reduce(nb, c, q2, p, part + 2 * (size_t)nb * c * p * p, act, RQ, st, srq);
  PC_CK_LAUNCH();
  return PC_OK;
}

// G = A^H B (complex64, p <= 64 columns of A, q <= 128 of B) on the tensor cores; PC_EUNSUPPORTED as above.
int launch_gram_tc(int nb, long L, int p, int q, const void *A, long sa, const void *B, long sb, void *G,
                   void *scratch, size_t scratch_bytes, cudaStream_t st, const int *act, int nb_alloc, long sg) {
  if (!tc_shape_ok(L, p, q, A, sa, B, sb)) return PC_EUNSUPPORTED;
  int c = 0;
  double2 *part = static_cast<double2 *>(scratch);
  // the wider panel takes the MMA rows (2 x its columns of the 128): B^H A, written conjugate-transposed
  const bool swap = q > p && q <= 64;
  int rc = swap ? launch_tc(nb, nb_alloc > 0 ? nb_alloc : nb, L, q, p, false, B, sb, A, sa, part, scratch_bytes, st,
                            act, &c, true)
                : launch_tc(nb, nb_alloc > 0 ? nb_alloc : nb, L, p, q, false, A, sa, B, sb, part, scratch_bytes, st,
                            act, &c);
  if (rc) return rc;
  launch_gram_reduce(nb, c, p, q, part, act, G, st, sg);
  PC_CK_LAUNCH();
  return PC_OK;
}

// reads and clears the abort flag of the tensor-core Gram kernel (after a synchronisation)
int gram_tc_check() {
  int v = 0;
  PC_CK(cudaMemcpyFromSymbol(&v, g_gram_tc_error, sizeof(int)));
  if (v) {
    const int zero = 0;
    PC_CK(cudaMemcpyToSymbol(g_gram_tc_error, &zero, sizeof(int)));
    set_error("tensor-core Gram kernel: a pipeline wait ran out of time");
    return PC_ECUDA;
  }
  return PC_OK;
}

}  // namespace pc
