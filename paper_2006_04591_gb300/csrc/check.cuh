// check.cuh - bounds guards of the checked build.
//
// Compiled with -DSHL_CHECKED, every guarded global access of the transform
// kernels first compares its index with the extent of the buffer it
// addresses (derived from the launch's own sizes); an index outside sets bit
// `code` of the translation unit's device word g_shl_check and the access
// is skipped (a load gives 0), so a wrong index shows up as a flag read by
// shl_check_status instead of a fault.  Without SHL_CHECKED the guards are
// constant true and vanish.
#pragma once

#include <stddef.h>

#ifdef SHL_CHECKED
#define SHL_CHECK_WORD_DEFINE __device__ unsigned int g_shl_check = 0;
#define SHL_IN(i, n, code) \
  (((size_t)(i) < (size_t)(n)) ? true : (atomicOr(&g_shl_check, (unsigned)(code)), false))
#else
#define SHL_CHECK_WORD_DEFINE
#define SHL_IN(i, n, code) true
#endif

namespace shl {
// Guard bits of the transform kernels.
enum CheckCode : unsigned {
  CHK_R2C_IN = 1u << 0, CHK_R2C_OUT = 1u << 1, CHK_C2R_IN = 1u << 2, CHK_C2R_OUT = 1u << 3,
  CHK_LINES = 1u << 4, CHK_DEC_X = 1u << 5, CHK_DEC_G = 1u << 6, CHK_DEC_OUT = 1u << 7,
  CHK_REC_STAGE = 1u << 8, CHK_REC_G = 1u << 9, CHK_REC_ACC = 1u << 10, CHK_SHRINK = 1u << 11,
  CHK_ABSMAX = 1u << 12,
  // tc_dft.cu
  CHK_TC_X = 1u << 13, CHK_TC_G = 1u << 14, CHK_TC_OUT = 1u << 15,
};
}  // namespace shl
