// Shared layout constants of the tensor-core H_eff path (heff_tc.cu, tc_host.cu).
#pragma once
#include <stdint.h>

namespace mrd {

// Tensor-core precisions: complex operands, or real ones (the sine / cosine machine of Eq. rot
// with real environments and theta: imaginary planes dropped, the result's imaginary parts 0).
enum { TC_TF32 = 1, TC_BF16X3 = 2, TC_TF32_REAL = 3, TC_BF16X3_REAL = 4 };
__host__ __device__ inline bool tc_is_tf32(int prec) { return prec == TC_TF32 || prec == TC_TF32_REAL; }
__host__ __device__ inline bool tc_is_real(int prec) { return prec == TC_TF32_REAL || prec == TC_BF16X3_REAL; }
// task row (int64): M N out0 out1 pad seg0 nseg mode nkt_z pad
//   mode 0: packed Z output, out0 = byte offset of the Z panel, nkt_z its K-tile count
//   mode 1: FP64 output, out0 = element offset, out1 = leading dimension
//   mode 2: packed Z output of stacked rows, out0 = first entry of the task in the row map
//           ((Z panel byte offset << 16) | row in that panel, one per output row), nkt_z the
//           K-tile count of those panels
enum { TCT = 10 };
// segment row: a_panel_byte_offset b_panel_byte_offset nkt pad
enum { TCS = 4 };
// pack job row: src_off ld trans rows K panel_byte_offset rowtile nkt npad first_piece format
// row0 k0, where the job's 16-byte chunks (rows x ceil(K / chunk K)) are cut into pieces of
// kPackPiece and first_piece is the prefix of the earlier jobs' pieces; format 0 writes the
// A planes, 1 the B planes; row0 / k0 place the block inside a larger panel (multiples of
// the chunk's K for k0)
enum { TCJ = 13 };
constexpr int kPackPiece = 1024;

// Planes of a packed tile. A operands (LW, Z): re, im (TF32) or re_hi, re_lo, im_hi, im_lo
// (split BF16). B operands (theta, WR) carry their imaginary planes negated as well, ordered
// so that two windows of consecutive planes are the B operands of one complex product:
//   TF32    S = [-im, re, im]:  C += A_re x S[1..2] + A_im x S[0..1]
//   BF16X3  S = [-im_hi, -im_lo, re_hi, re_lo, im_hi, im_lo]:
//           C += (A_re_hi + A_re_lo) x S[2..5] + (A_im_hi + A_im_lo) x S[0..3]
// The accumulator then holds the column groups (re, im) or (re_hi, re_lo, im_hi, im_lo) of
// the output side by side, and the epilogue adds each part's pieces.
// Real operands: A and B both [re] (TF32) or [re_hi, re_lo] (BF16X3), C[hi | lo] += A_hi x
// [hi | lo] + A_lo x [hi | lo] (2 MMAs of N = 2 nrow; 1 MMA of N = nrow for TF32).
__host__ __device__ inline int tc_aplanes(int prec) {
  return prec == TC_TF32 ? 2 : prec == TC_BF16X3 ? 4 : prec == TC_TF32_REAL ? 1 : 2;
}
__host__ __device__ inline int tc_bplanes(int prec) {
  return prec == TC_TF32 ? 3 : prec == TC_BF16X3 ? 6 : prec == TC_TF32_REAL ? 1 : 2;
}
// accumulator column groups of one output tile (one per B plane of a window)
__host__ __device__ inline int tc_groups(int prec) {
  return prec == TC_TF32 ? 2 : prec == TC_BF16X3 ? 4 : prec == TC_TF32_REAL ? 1 : 2;
}
__host__ __device__ inline int tc_kpt(int prec) { return tc_is_tf32(prec) ? 32 : 64; }   // K per 128-byte row
// Tile configuration of the grouped GEMM, picked per problem class by the autotuner
// (tc_host.cu): B rows (output columns) per tile, pipeline stages, task order (0: charge
// order, 1: largest work first).
struct TcCfg {
  int ntile, stages, order;
};
constexpr int kTcMaxStages = 4;
// dynamic shared memory; with the kernel's ~120 bytes of static shared memory it stays below
// the 227 KB a block may use
constexpr int kTcMaxSmem = 225 * 1024;
// shared-memory stage: A planes x 16 KB + B planes x ntile x 128 B
__host__ __device__ inline int tc_stage_bytes(int prec, int ntile) {
  return tc_aplanes(prec) * 128 * 128 + tc_bplanes(prec) * ntile * 128;
}
__host__ __device__ inline int tc_smem_bytes(int prec, TcCfg c) { return c.stages * tc_stage_bytes(prec, c.ntile) + 1024; }
// the accumulator of one tile spans groups x ntile FP32 columns: at most 256, so that two
// tiles (two slots) fit the 512 columns of tensor memory
__host__ __device__ inline bool tc_cfg_ok(int prec, TcCfg c) {
  return c.stages >= 1 && c.stages <= kTcMaxStages && c.ntile >= 16 && c.ntile % 16 == 0 &&
         tc_groups(prec) * c.ntile <= 256 && tc_smem_bytes(prec, c) <= kTcMaxSmem;
}
// default configuration (also the first candidate of the autotuner)
inline TcCfg tc_default_cfg(int prec) {
  return prec == TC_TF32 ? TcCfg{128, 2, 0} : prec == TC_BF16X3 ? TcCfg{64, 2, 0} : TcCfg{128, 3, 0};
}

}  // namespace mrd
