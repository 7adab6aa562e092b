// Shared layout constants of the tensor-core H_eff path (heff_tc.cu, tc_host.cu).
#pragma once
#include <stdint.h>

namespace mrd {

enum { TC_TF32 = 1, TC_BF16X3 = 2 };
// task row (int64): M N out0 out1 pad seg0 nseg mode nkt_z pad
//   mode 0: packed Z output, out0 = byte offset of the Z panel, nkt_z its K-tile count
//   mode 1: FP64 output, out0 = element offset, out1 = leading dimension
enum { TCT = 10 };
// segment row: a_panel_byte_offset b_panel_byte_offset nkt pad
enum { TCS = 4 };
// pack job row: src_off ld trans rows K panel_byte_offset rowtile nkt npad first_piece, where
// the job's 16-byte chunks (rows x ceil(K / chunk K)) are cut into pieces of kPackPiece and
// first_piece is the prefix of the earlier jobs' pieces
enum { TCJ = 10 };
constexpr int kPackPiece = 1024;

struct TcPanelGeom {
  int64_t nkt;
  int planes;
};

__host__ __device__ inline int tc_planes(int prec) { return prec == TC_TF32 ? 2 : 4; }
__host__ __device__ inline int tc_kpt(int prec) { return prec == TC_TF32 ? 32 : 64; }   // K per 128-byte row
// Tile configuration of the grouped GEMM, picked per problem class by the autotuner
// (tc_host.cu): B rows (output columns) per tile, pipeline stages, task order (0: charge
// order, 1: largest work first).
struct TcCfg {
  int ntile, stages, order;
};
constexpr int kTcMaxStages = 4;
constexpr int kTcMaxSmem = 220 * 1024;   // dynamic; the kernel's static shared memory comes on top
// shared-memory stage: A planes x 16 KB + B planes x ntile x 128 B
__host__ __device__ inline int tc_stage_bytes(int prec, int ntile) {
  return tc_planes(prec) * (128 * 128 + ntile * 128);
}
__host__ __device__ inline int tc_smem_bytes(int prec, TcCfg c) { return c.stages * tc_stage_bytes(prec, c.ntile) + 1024; }
// default configuration (also the first candidate of the autotuner)
inline TcCfg tc_default_cfg(int prec) { return prec == TC_TF32 ? TcCfg{128, 3, 0} : TcCfg{64, 2, 0}; }

}  // namespace mrd
