// Host-side argument checks shared by the entry points.
#pragma once
#include "fa.h"

namespace fa {
fa_status check_vol(const fa_vol *v, const char *name, int C);
fa_status same_grid(const fa_vol *a, const fa_vol *b, const char *an, const char *bn);
fa_status check_ws(const void *ws, size_t have, size_t need, const char *who);
}  // namespace fa
