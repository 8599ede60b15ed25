// Host-side argument checks shared by the entry points.
#pragma once
#include "fa.h"

namespace fa {
fa_status check_vol(const fa_vol *v, const char *name, int C);
// check_vol for a volume of element type `dtype` (FA_F32, FA_BF16 or FA_F16).
fa_status check_vol_dtype(const fa_vol *v, const char *name, int C, int dtype);
fa_status same_grid(const fa_vol *a, const fa_vol *b, const char *an, const char *bn);
fa_status check_ws(const void *ws, size_t have, size_t need, const char *who);
}  // namespace fa
