// Charge bookkeeping of one two-site problem, built on the device (see plan.cu).
#pragma once
#include <stdint.h>

namespace mrd {

// Row widths of the int64 tables.
enum { MIDF = 12, LWF = 10, WRF = 10, ZF = 6, TF = 6, SF = 6 };
// MID row: N K rowdim coldim offset row_a0 row_a1 row_off1 col_b0 col_b1 col_off1 pad
// LW row : w' s1' s1 a a' rows cols offset contrib_begin contrib_end
// WR row : w' s2 s2' b b' rows cols offset contrib_begin contrib_end
// Z row  : w' m_in m_out rows cols offset
// task   : M N c_off ldc seg_begin seg_count
// segment: a_off lda b_off ldb K flags (bit 0: A conjugate-transposed, bit 1: B conjugate-transposed)
enum Count {
  C_NMID = 0, C_THETA, C_LENV, C_RENV, C_NLW, C_LWLEN, C_NWR, C_WRLEN, C_NZ, C_ZLEN,
  C_NT1, C_NT2, C_TILES1, C_TILES2, C_FLOPS1, C_FLOPS2, C_ERR, C_NCOUNTS
};

struct PlanDims {
  int32_t n_l, n_r, d_l, d_m, d_r, nnz_i, nnz_j, m1, m2, mod;
  int64_t mid_cap, lw_cap, wr_cap, z_cap, t1_cap, t2_cap, seg2_stride, scratch_len;
};

struct PlanPtrs {
  const int32_t *left, *right, *cl, *cm, *cr, *wi_idx, *wj_idx;
  int32_t *wi_perm, *wj_perm;   // entry order sorted by (w', s1', s1, w) / (w', s2, s2', w'')
  int32_t *trip_i, *trip_j;     // per (w', x, y): [begin, end) into the sorted order
  int64_t *mid, *counts, *lmap, *rmap, *lwmap, *lw, *wrmap, *wr, *zmap, *z;
  int32_t *s1mask;
  int64_t *t1, *seg1, *tile1, *t2, *seg2, *tile2;
  int64_t *scr_a, *scr_b;
};

}  // namespace mrd
