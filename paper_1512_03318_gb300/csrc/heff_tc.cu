// Tensor-core (tcgen05 / TMEM) grouped complex GEMMs of the two-site H_eff in reduced
// precision with FP32 accumulation.
//
// Same two steps as the FP64 path (step 1: Z_{w'} = LW_{w'} theta; step 2:
// theta' = sum_{w'} Z_{w'} WR_{w'}), same task decomposition. A complex product is four real
// products on real tensor cores, C_re = A_re B_re - A_im B_im and C_im = A_re B_im + A_im B_re,
// the minus sign coming from the A-negate bit of the instruction descriptor. Precisions:
//   TF32    operands rounded to TF32 (planes re, im); 4 MMAs per complex product step.
//   BF16X3  every operand x split as x_hi = bf16(x), x_lo = bf16(x - x_hi) (planes re_hi,
//           re_lo, im_hi, im_lo); A_hi B_hi + A_hi B_lo + A_lo B_hi per real product, so 12
//           MMAs per complex step (the split-precision scheme of Henry, Tang & Heinecke 2019).
//
// Operands live in HBM as "panels" of UMMA-ready tiles: a tile is R rows x 128 bytes of K
// (32 TF32 or 64 BF16 values), K-major, 128-byte swizzled, zero padded, with its planes
// stored back to back, so one cp.async.bulk moves a tile into shared memory unchanged.
// A panels have 128-row tiles; B panels hold all N rows (padded to 16), 128 (TF32) or 64
// (BF16) rows per tile.
// LW and WR are packed once per environment load, theta once per matvec, and the step-1
// epilogue writes Z directly in the packed A format of step 2.
//
// Kernel: persistent, one CTA per SM, 6 warps: warp 0 issues the bulk copies, warp 1 owns
// TMEM (512 columns: two accumulator slots of C_re, C_im) and issues the MMAs from one thread, warps 2-5
// drain the accumulators (warp w reads TMEM lanes 32 (w % 4) ..). Shared-memory stages are
// handed over with mbarriers; every wait is bounded (global-timer limit set by the host) and
// sets an error flag when it gives up. Before the CTA frees its tensor memory and exits, the
// producer waits for the last fill of every stage and the MMA thread for all its MMAs (commit
// to a drain barrier), so a CTA whose waits gave up leaves no copy or MMA in flight.
#include <cuda_bf16.h>

#include "mrd_internal.h"
#include "tc.cuh"

namespace mrd {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t sw128(uint32_t row, uint32_t byte_in_row) {
  const uint32_t lin = row * 128u + byte_in_row;
  return lin ^ (((lin >> 7) & 7u) << 4);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // SBO: 8 rows x 128 bytes
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

__device__ __forceinline__ uint32_t make_idesc(int prec, int n, bool neg_a) {
  uint32_t d = 0;
  d |= 1u << 4;                                        // D: FP32
  if (tc_is_tf32(prec)) { d |= 2u << 7; d |= 2u << 10; }  // A, B: TF32
  else { d |= 1u << 7; d |= 1u << 10; }                // A, B: BF16
  if (neg_a) d |= 1u << 13;
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(128 >> 4) << 24;
  return d;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t mbar_probe(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done;
}

// Wait for the phase of `parity` of an mbarrier to complete, for at most limit_ns nanoseconds
// of the global timer; limit_ns = 0 gives up without probing. On giving up, records `code` in
// the error flag (first failure wins) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, uint64_t limit_ns) {
  if (limit_ns > 0) {
    if (mbar_probe(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < limit_ns)
      if (mbar_probe(bar, parity)) return true;
  }
  atomicCAS(err, 0, code);
  return false;
}

// Limit of the waits that drain a CTA's own copies and MMAs before it frees its tensor memory
// and exits, whatever limit the work's waits had.
constexpr uint64_t kDrainNs = 2000000000ull;

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// The MMAs of one K step of a complex product, issued from one asm block with the accumulate
// predicate set once (acc = 0 starts the accumulator of the tile). Each MMA multiplies one A
// plane by a window of consecutive B planes (tc.cuh), so that its N spans every column group
// of the output at once: TF32 C[re | im] += A_re x [re | im] + A_im x [-im | re] (2 MMAs of
// N = 2 nrow); split BF16 C[re_hi | re_lo | im_hi | im_lo] += (A_re_hi + A_re_lo) x
// [re_hi | re_lo | im_hi | im_lo] + (A_im_hi + A_im_lo) x [-im_hi | -im_lo | re_hi | re_lo]
// (4 MMAs of N = 4 nrow; the lo x lo product comes with the windows and is kept).
__device__ __forceinline__ void mma_cplx_tf32(uint32_t tacc, uint64_t a_re, uint64_t a_im, uint64_t b_s0,
                                              uint64_t b_s1, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.b32 p, %5, 0;\nsetp.eq.b32 q, 0, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %4, %6, p;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %2, %3, %6, q;\n}\n"
      ::"r"(tacc), "l"(a_re), "l"(a_im), "l"(b_s0), "l"(b_s1), "r"(acc), "r"(idesc));
}

__device__ __forceinline__ void mma_cplx_bf16x3(uint32_t tacc, uint64_t a_rh, uint64_t a_rl, uint64_t a_ih,
                                                uint64_t a_il, uint64_t b_s0, uint64_t b_s2, uint32_t idesc,
                                                uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.b32 p, %7, 0;\nsetp.eq.b32 q, 0, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %6, %8, p;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %6, %8, q;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %5, %8, q;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %5, %8, q;\n}\n"
      ::"r"(tacc), "l"(a_rh), "l"(a_rl), "l"(a_ih), "l"(a_il), "l"(b_s0), "l"(b_s2), "r"(acc), "r"(idesc));
}

// Real operands: TF32 C[re] += A x B (1 MMA of N = nrow); split BF16 C[hi | lo] +=
// (A_hi + A_lo) x [B_hi | B_lo] (2 MMAs of N = 2 nrow, the four products of the split).
__device__ __forceinline__ void mma_real_tf32(uint32_t tacc, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %3, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %4, p;\n}\n"
      ::"r"(tacc), "l"(a), "l"(b), "r"(acc), "r"(idesc));
}

__device__ __forceinline__ void mma_real_bf16x3(uint32_t tacc, uint64_t a_hi, uint64_t a_lo, uint64_t b,
                                                uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.b32 p, %4, 0;\nsetp.eq.b32 q, 0, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %5, p;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %3, %5, q;\n}\n"
      ::"r"(tacc), "l"(a_hi), "l"(a_lo), "l"(b), "r"(acc), "r"(idesc));
}

// 16 consecutive FP32 columns of the warp's 32 TMEM lanes (one row per lane); the caller waits
// with tcgen05.wait::ld before reading the registers.
__device__ __forceinline__ void tmem_ld16(uint32_t* v, uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                 "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
               : "r"(taddr));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ int64_t find_task(const int64_t* prefix, int64_t n, int64_t item) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace

// ---------------------------------------------------------------- packing kernels

// Pack FP64 complex blocks into panels. Each job: src element offset, src row stride,
// transpose flag (0: panel row r, col k = src[r * ld + k]; 1: = src[k * ld + r]), rows, K,
// destination panel byte offset, row tile height (128 for A, the tile column count for B), nkt,
// padded panel rows, first piece, format (0: A planes, 1: B planes with the negated imaginary
// parts), and the block's first row and first K inside the panel (row0, k0; k0 a multiple of
// the chunk's K). One thread writes one 16-byte chunk of a panel row in every plane: 4
// consecutive K values (TF32) or 8 (BF16). For transposed sources consecutive threads take
// consecutive panel rows, so each of the chunk's reads is coalesced; K beyond the block is
// written as zero padding. A CTA takes one piece (kPackPiece chunks of one job) at a time, so
// large blocks spread over the whole grid. The BF16 split is done in FP32 after one
// conversion of each value (hi = bf16(x), lo = bf16(x - hi), with x - hi exact in FP32): the
// split's error, ~2^-17 |x| from rounding lo, is the same as splitting in FP64, and the FP64
// pipe (2 ops per clock per SM) only converts. Negation is exact in both formats.
__global__ void k_pack(const double2* __restrict__ src, uint8_t* __restrict__ dst, const int64_t* __restrict__ jobs,
                       int njobs, int64_t npieces, int prec) {
  const bool tf32 = tc_is_tf32(prec), real = tc_is_real(prec);
  const int kc = tf32 ? 4 : 8;                   // K values per 16-byte chunk
  const int kpt = tf32 ? 32 : 64;                // K values per 128-byte row
  for (int64_t pc = blockIdx.x; pc < npieces; pc += gridDim.x) {
    int lo = 0, hi = njobs - 1;                  // the last job whose first piece is <= pc
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[TCJ * mid + 9] <= pc) lo = mid; else hi = mid - 1;
    }
    const int64_t* d = jobs + TCJ * lo;
    const int64_t s_off = d[0], ld = d[1], trans = d[2], rows = d[3], K = d[4], p_off = d[5], rowtile = d[6],
                  nkt = d[7], npad = d[8], bfmt = d[10], row0 = d[11], kbase = d[12];
    const int planes = bfmt ? tc_bplanes(prec) : tc_aplanes(prec);
    const int64_t nch = (K + kc - 1) / kc;       // chunks per row
    const int64_t e0 = (pc - d[9]) * kPackPiece;
    const int64_t e1 = e0 + kPackPiece < rows * nch ? e0 + kPackPiece : rows * nch;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      int64_t r, ch;
      if (trans) { ch = e / rows; r = e % rows; }   // consecutive threads: consecutive rows
      else { r = e / nch; ch = e % nch; }           // consecutive threads: consecutive chunks
      const int64_t k0 = ch * kc;                   // within the block
      const int64_t pr = row0 + r, pk = kbase + k0; // within the panel
      const int64_t rt = pr / rowtile, kt = pk / kpt;
      const int64_t nrow = npad - rt * rowtile < rowtile ? npad - rt * rowtile : rowtile;
      const int64_t tile_bytes = nrow * 128;       // one plane of this row tile
      uint8_t* tile = dst + p_off + rt * nkt * planes * rowtile * 128 + kt * planes * tile_bytes;
      const uint32_t off = sw128((uint32_t)(pr % rowtile), (uint32_t)((pk % kpt) * (tf32 ? 4 : 2)));
      if (tf32) {
        float4 re, im;
        float* pre = (float*)&re;
        float* pim = (float*)&im;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t k = k0 + q;
          double2 v = make_double2(0.0, 0.0);
          if (k < K) v = trans ? src[s_off + k * ld + r] : src[s_off + r * ld + k];
          pre[q] = tf32_rna((float)v.x);
          pim[q] = tf32_rna((float)v.y);
        }
        if (real) {    // [re]
          *(float4*)(tile + off) = re;
        } else if (bfmt) {    // [-im, re, im]
          const float4 nim = make_float4(-im.x, -im.y, -im.z, -im.w);
          *(float4*)(tile + off) = nim;
          *(float4*)(tile + tile_bytes + off) = re;
          *(float4*)(tile + 2 * tile_bytes + off) = im;
        } else {       // [re, im]
          *(float4*)(tile + off) = re;
          *(float4*)(tile + tile_bytes + off) = im;
        }
      } else {
        uint4 pl[6];   // re_hi, re_lo, im_hi, im_lo, -im_hi, -im_lo
        __nv_bfloat16* b[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) b[q] = (__nv_bfloat16*)&pl[q];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t k = k0 + q;
          double2 v = make_double2(0.0, 0.0);
          if (k < K) v = trans ? src[s_off + k * ld + r] : src[s_off + r * ld + k];
          const float xr = __double2float_rn(v.x), xi = __double2float_rn(v.y);
          const __nv_bfloat16 rh = __float2bfloat16_rn(xr);
          const __nv_bfloat16 ih = __float2bfloat16_rn(xi);
          const __nv_bfloat16 rl = __float2bfloat16_rn(__fsub_rn(xr, __bfloat162float(rh)));
          const __nv_bfloat16 il = __float2bfloat16_rn(__fsub_rn(xi, __bfloat162float(ih)));
          b[0][q] = rh;
          b[1][q] = rl;
          b[2][q] = ih;
          b[3][q] = il;
          b[4][q] = __hneg(ih);
          b[5][q] = __hneg(il);
        }
        if (real) {    // [re_hi, re_lo]
          *(uint4*)(tile + off) = pl[0];
          *(uint4*)(tile + tile_bytes + off) = pl[1];
        } else if (bfmt) {    // [-im_hi, -im_lo, re_hi, re_lo, im_hi, im_lo]
          const int order[6] = {4, 5, 0, 1, 2, 3};
#pragma unroll
          for (int q = 0; q < 6; ++q) *(uint4*)(tile + q * tile_bytes + off) = pl[order[q]];
        } else {       // [re_hi, re_lo, im_hi, im_lo]
#pragma unroll
          for (int q = 0; q < 4; ++q) *(uint4*)(tile + q * tile_bytes + off) = pl[q];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- grouped GEMM

struct TcArgs {
  const uint8_t* a_base;   // packed A panels
  const uint8_t* b_base;   // packed B panels
  const int64_t* tasks;    // TCT per task
  const int64_t* segs;     // TCS per segment
  const int64_t* prefix;   // tiles prefix (n_tasks + 1)
  int64_t n_tasks;
  uint8_t* z_out;          // packed Z output (mode 0)
  double2* f_out;          // FP64 output (mode 1)
  int prec;
  int* err;
  const int2* items;       // per tile item: (task, tile within the task), or null: search the prefix
  const int32_t* cta_off;  // with items: CTA c runs items cta_off[c] .. cta_off[c + 1] - 1; null:
                           // items blockIdx.x, + gridDim.x, ...
  int ntile;               // B rows per tile (multiple of 16, at most 128)
  int nstages;             // shared-memory pipeline depth (at most kTcMaxStages)
  int stage_bytes;
  uint64_t wait_ns;        // limit of each pipeline wait (ns); 0: the first wait gives up
  const int64_t* rowmap;   // mode 2: per output row (Z panel byte offset << 16) | row in that panel
};

// Task and tile of a work item: one load from the host-built item table, else a binary
// search over the tile prefix (per-task launches, one task).
__device__ __forceinline__ void item_of(const TcArgs& g, int64_t item, int64_t& t, int64_t& local) {
  if (g.items) {
    const int2 v = g.items[item];
    t = v.x;
    local = v.y;
  } else {
    t = find_task(g.prefix, g.n_tasks, item);
    local = item - g.prefix[t];
  }
}

// Accumulator slots in TMEM: slot b holds C_re at columns 256 b and C_im at 256 b + 128.
constexpr int kAccSlots = 2;

// Write 16 consecutive output values of one row into a packed panel (16-byte chunks).
__device__ __forceinline__ void put_packed16(uint8_t* base, int64_t nkt, int planes, int prec, int64_t row,
                                             int64_t k0, const float* re, const float* im, int nvalid) {
  const int kpt = tc_kpt(prec);
  const int64_t rt = row / 128, kt = k0 / kpt;
  uint8_t* tile = base + (rt * nkt + kt) * planes * (int64_t)(128 * 128);
  const uint32_t r = (uint32_t)(row % 128);
  const int kin = (int)(k0 % kpt);
  const bool real = tc_is_real(prec);
  if (tc_is_tf32(prec)) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {          // 4 chunks of 4 TF32 values
      uint4 vr, vi;
      float* fr = (float*)&vr;
      float* fi = (float*)&vi;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 4 * q + e;
        fr[e] = j < nvalid ? tf32_rna(re[j]) : 0.f;
        fi[e] = j < nvalid ? tf32_rna(im[j]) : 0.f;
      }
      const uint32_t off = sw128(r, (uint32_t)((kin + 4 * q) * 4));
      *(uint4*)(tile + off) = vr;
      if (!real) *(uint4*)(tile + 128 * 128 + off) = vi;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 2; ++q) {          // 2 chunks of 8 BF16 values per plane
      uint4 v[4];
      __nv_bfloat16* b[4];
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) b[pl] = (__nv_bfloat16*)&v[pl];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = 8 * q + e;
        const float x = j < nvalid ? re[j] : 0.f, y = j < nvalid ? im[j] : 0.f;
        const __nv_bfloat16 xh = __float2bfloat16_rn(x), yh = __float2bfloat16_rn(y);
        b[0][e] = xh;
        b[1][e] = __float2bfloat16_rn(x - __bfloat162float(xh));
        b[2][e] = yh;
        b[3][e] = __float2bfloat16_rn(y - __bfloat162float(yh));
      }
      const uint32_t off = sw128(r, (uint32_t)((kin + 8 * q) * 2));
#pragma unroll
      for (int pl = 0; pl < 4; ++pl)
        if (!real || pl < 2) *(uint4*)(tile + pl * 128 * 128 + off) = v[pl];   // real: [hi, lo]
    }
  }
}

__global__ void __launch_bounds__(192, 1) k_tc_gemm(TcArgs g) {
  extern __shared__ uint8_t dyn[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[kTcMaxStages], bar_empty[kTcMaxStages], bar_acc_full[kAccSlots],
      bar_acc_empty[kAccSlots], bar_drain;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int prec = g.prec;
  const int aplanes = tc_aplanes(prec), bplanes = tc_bplanes(prec), groups = tc_groups(prec);
  const int kpt = tc_kpt(prec);                    // K values per 128-byte row
  const int kstep = tc_is_tf32(prec) ? 8 : 16;     // K per MMA instruction
  const int ntile = g.ntile;                       // B rows (output columns) per tile
  const int nstages = g.nstages;
  const int stage_bytes = g.stage_bytes;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < kAccSlots; ++b) {
      mbar_init(smem_u32(&bar_acc_full[b]), 1);
      mbar_init(smem_u32(&bar_acc_empty[b]), 4);
    }
    mbar_init(smem_u32(&bar_drain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int64_t total = g.prefix[g.n_tasks];
  // this CTA's work items: its own list (host-balanced deal) or every gridDim.x-th item; the
  // producer, the MMA thread and the epilogue walk the same sequence
  const bool listed = g.items != nullptr && g.cta_off != nullptr;
  const int64_t it_first = listed ? (int64_t)g.cta_off[blockIdx.x] : (int64_t)blockIdx.x;
  const int64_t it_last = listed ? (int64_t)g.cta_off[blockIdx.x + 1] : total;
  const int64_t it_step = listed ? 1 : (int64_t)gridDim.x;

  if (warp == 0 && lane == 0) {
    // ---------------- producer
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    int64_t fills = 0;   // stage fills issued
    for (int64_t item = it_first, it_end = it_last; item < it_end && ok; item += it_step) {
      int64_t t, local;
      item_of(g, item, t, local);
      const int64_t* task = g.tasks + TCT * t;
      const int64_t N = task[1];
      const int64_t tiles_n = (N + ntile - 1) / ntile;
      const int64_t rt = local / tiles_n, nt = local % tiles_n;
      const int64_t npad = ((N + 15) / 16) * 16;
      const int64_t nrow = npad - nt * ntile < ntile ? npad - nt * ntile : ntile;
      // rows of this A row tile that hold data, rounded up to a swizzle atom of 8 rows: only
      // these are copied; the stage's other rows keep stale values, which reach only
      // accumulator rows the epilogue never stores
      const int64_t mleft = task[0] - rt * 128;
      const uint32_t mrows = (uint32_t)(((mleft < 128 ? mleft : 128) + 7) / 8 * 8);
      for (int64_t s = 0; s < task[6] && ok; ++s) {
        const int64_t* sg = g.segs + TCS * (task[5] + s);
        const int64_t nkt = sg[2];
        const uint8_t* a = g.a_base + sg[0] + rt * nkt * aplanes * (int64_t)(128 * 128);
        const uint8_t* b = g.b_base + sg[1] + nt * nkt * bplanes * (int64_t)ntile * 128;
        for (int64_t kt = 0; kt < nkt && ok; ++kt) {
          ok = mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1, g.err, 11, g.wait_ns);
          if (!ok) break;
          const uint32_t abytes = aplanes * 128 * 128, bbytes = (uint32_t)(bplanes * nrow * 128);
          const uint32_t sa = smem_u32(smem + stage * stage_bytes);
          const uint32_t sb = sa + abytes;
          mbar_expect_tx(smem_u32(&bar_full[stage]), (uint32_t)aplanes * mrows * 128 + bbytes);
          for (int p = 0; p < aplanes; ++p)
            bulk_g2s(sa + p * 128 * 128, a + kt * abytes + p * 128 * 128, mrows * 128, smem_u32(&bar_full[stage]));
          bulk_g2s(sb, b + kt * (int64_t)bbytes, bbytes, smem_u32(&bar_full[stage]));
          ++fills;
          if (++stage == nstages) { stage = 0; phase ^= 1; }
        }
      }
    }
    // drain: the last fills of every stage have landed before the CTA may exit (after normal
    // work they have, since the MMAs consumed them; after a wait gave up they may not have)
    for (int64_t f = fills - 1; f >= 0 && f >= fills - nstages; --f)
      mbar_wait(smem_u32(&bar_full[f % nstages]), (uint32_t)((f / nstages) & 1), g.err, 15, kDrainNs);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int stage = 0;
    uint32_t phase = 0;
    uint32_t acc_phase = 0;   // bit b: phase of slot b
    int slot = 0;
    bool ok = true;
    for (int64_t item = it_first, it_end = it_last; item < it_end && ok; item += it_step) {
      int64_t t, local;
      item_of(g, item, t, local);
      const int64_t* task = g.tasks + TCT * t;
      const int64_t N = task[1];
      const int64_t tiles_n = (N + ntile - 1) / ntile;
      const int64_t nt = local % tiles_n;
      const int64_t npad = ((N + 15) / 16) * 16;
      const int nrow = (int)(npad - nt * ntile < ntile ? npad - nt * ntile : ntile);
      ok = mbar_wait(smem_u32(&bar_acc_empty[slot]), ((acc_phase >> slot) & 1) ^ 1, g.err, 12, g.wait_ns);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t tacc = tmem + 256 * slot;   // groups x nrow <= 256 columns
      const uint32_t idesc = make_idesc(prec, groups * nrow, false);
      bool first = true;
      for (int64_t s = 0; s < task[6] && ok; ++s) {
        const int64_t nkt = g.segs[TCS * (task[5] + s) + 2];
        for (int64_t kt = 0; kt < nkt && ok; ++kt) {
          ok = mbar_wait(smem_u32(&bar_full[stage]), phase, g.err, 13, g.wait_ns);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t sa = smem_u32(smem + stage * stage_bytes);
          const uint32_t sb = sa + aplanes * 128 * 128;
          // descriptors of the stage's planes; a K step of 32 bytes adds 2 to the address field
          // (smem address / 16 in bits 0-13, no carry below 256 KB), so each instruction's
          // descriptors are one 64-bit add away from these
          const uint64_t a0 = make_desc(sa), b0 = make_desc(sb);
          const uint64_t pa = (128 * 128) >> 4, pb = ((uint32_t)nrow * 128) >> 4;
          const int nks = kpt / kstep;
          for (int ks = 0; ks < nks; ++ks) {
            const uint64_t ko = 2 * ks;
            const uint32_t acc = first ? 0u : 1u;
            if (prec == TC_TF32)
              mma_cplx_tf32(tacc, a0 + ko, a0 + pa + ko, b0 + ko, b0 + pb + ko, idesc, acc);
            else if (prec == TC_BF16X3)
              mma_cplx_bf16x3(tacc, a0 + ko, a0 + pa + ko, a0 + 2 * pa + ko, a0 + 3 * pa + ko, b0 + ko,
                              b0 + 2 * pb + ko, idesc, acc);
            else if (prec == TC_TF32_REAL)
              mma_real_tf32(tacc, a0 + ko, b0 + ko, idesc, acc);
            else
              mma_real_bf16x3(tacc, a0 + ko, a0 + pa + ko, b0 + ko, idesc, acc);
            first = false;
          }
          mma_commit(smem_u32(&bar_empty[stage]));
          if (++stage == nstages) { stage = 0; phase ^= 1; }
        }
      }
      mma_commit(smem_u32(&bar_acc_full[slot]));
      acc_phase ^= 1u << slot;
      slot ^= 1;
    }
    // drain: every MMA this thread issued has completed before the tensor memory is freed
    mma_commit(smem_u32(&bar_drain));
    mbar_wait(smem_u32(&bar_drain), 0, g.err, 16, kDrainNs);
  } else if (warp >= 2) {
    // ---------------- epilogue
    const int quad = warp & 3;            // TMEM lanes 32*quad .. 32*quad+31
    uint32_t acc_phase = 0;   // bit b: phase of slot b
    int slot = 0;
    bool ok = true;
    for (int64_t item = it_first, it_end = it_last; item < it_end && ok; item += it_step) {
      int64_t t, local;
      item_of(g, item, t, local);
      const int64_t* task = g.tasks + TCT * t;
      const int64_t M = task[0], N = task[1];
      const int64_t tiles_n = (N + ntile - 1) / ntile;
      const int64_t rt = local / tiles_n, nt = local % tiles_n;
      ok = mbar_wait(smem_u32(&bar_acc_full[slot]), (acc_phase >> slot) & 1, g.err, 14, g.wait_ns);
      acc_phase ^= 1u << slot;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t row = rt * 128 + quad * 32 + lane;
      const int64_t c0 = nt * ntile;
      const int64_t ncols = N - c0 < ntile ? N - c0 : ntile;
      const uint32_t tacc = tmem + 256 * slot + ((uint32_t)(quad * 32) << 16);
      const int64_t npad = ((N + 15) / 16) * 16;
      const uint32_t nrow = (uint32_t)(npad - c0 < ntile ? npad - c0 : ntile);   // columns of a group
      for (int64_t cb = 0; cb < ncols; cb += 16) {
        // group g of the accumulator sits at columns g * nrow; split BF16 adds the hi and lo
        // groups of each part
        uint32_t vr[16], vi[16], wr[16], wi[16];
        const uint32_t c = (uint32_t)cb;
        const bool real = tc_is_real(prec);
        if (real) {                 // [re] or [re_hi | re_lo]
          tmem_ld16(vr, tacc + c);
          if (groups == 2) tmem_ld16(wr, tacc + nrow + c);
        } else if (groups == 2) {   // [re | im]
          tmem_ld16(vr, tacc + c);
          tmem_ld16(vi, tacc + nrow + c);
        } else {                    // [re_hi | re_lo | im_hi | im_lo]
          tmem_ld16(vr, tacc + c);
          tmem_ld16(wr, tacc + nrow + c);
          tmem_ld16(vi, tacc + 2 * nrow + c);
          tmem_ld16(wi, tacc + 3 * nrow + c);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (row < M) {
          const int nvalid = (int)(ncols - cb < 16 ? ncols - cb : 16);
          float re[16], im[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            re[j] = __uint_as_float(vr[j]);
            im[j] = real ? 0.f : __uint_as_float(vi[j]);
          }
          if (real && groups == 2) {
#pragma unroll
            for (int j = 0; j < 16; ++j) re[j] = __fadd_rn(re[j], __uint_as_float(wr[j]));
          } else if (groups == 4) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              re[j] = __fadd_rn(re[j], __uint_as_float(wr[j]));
              im[j] = __fadd_rn(im[j], __uint_as_float(wi[j]));
            }
          }
          const int64_t col = c0 + cb;
          if (task[7] == 1) {
            double2* dst = g.f_out + task[2] + row * task[3] + col;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (j < nvalid) dst[j] = make_double2((double)re[j], (double)im[j]);
          } else if (task[7] == 2) {   // stacked rows: each goes to its own Z panel
            const int64_t rm = g.rowmap[task[2] + row];
            put_packed16(g.z_out + (rm >> 16), task[8], aplanes, prec, rm & 0xffff, col, re, im, nvalid);
          } else {
            put_packed16(g.z_out + task[2], task[8], aplanes, prec, row, col, re, im, nvalid);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty[slot]));
      slot ^= 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Kernel attributes (dynamic shared memory above 48 KB); called before any capture.
cudaError_t tc_gemm_init() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcMaxSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

cudaError_t tc_pack(const double2* src, uint8_t* dst, const int64_t* jobs, int njobs, int64_t npieces, int prec,
                    cudaStream_t s) {
  if (njobs <= 0 || npieces <= 0) return cudaSuccess;
  k_pack<<<(unsigned)(npieces < 8192 ? npieces : 8192), 256, 0, s>>>(src, dst, jobs, njobs, npieces, prec);
  mrd::count_launch();
  return cudaGetLastError();
}

cudaError_t tc_gemm(const uint8_t* a_base, const uint8_t* b_base, const int64_t* tasks, const int64_t* segs,
                    const int64_t* prefix, const int2* items, const int32_t* cta_off, const int64_t* rowmap,
                    int64_t n_tasks, int64_t total_tiles, uint8_t* z_out, double2* f_out, int prec, TcCfg cfg,
                    int* err, int n_sm, uint64_t wait_ns, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  cudaError_t ea = tc_gemm_init();
  if (ea != cudaSuccess) return ea;
  const int smem = tc_smem_bytes(prec, cfg);
  if (!tc_cfg_ok(prec, cfg) || smem > kTcMaxSmem) return cudaErrorInvalidValue;
  TcArgs g{a_base, b_base, tasks, segs, prefix, n_tasks, z_out, f_out, prec, err, items, cta_off, cfg.ntile, cfg.stages,
           tc_stage_bytes(prec, cfg.ntile), wait_ns, rowmap};
  const int64_t grid = total_tiles < n_sm ? total_tiles : n_sm;
  k_tc_gemm<<<(unsigned)grid, 192, smem, s>>>(g);
  mrd::count_launch();
  return cudaGetLastError();
}

}  // namespace mrd
