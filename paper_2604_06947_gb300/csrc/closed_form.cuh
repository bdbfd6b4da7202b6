// closed_form.cuh -- the integer closed form of a linear transfer map.
//
// For a linear split flux the table of eq. flux_table can coincide, on the
// whole visited range, with phi(q) = R(q*num/den) for small integers num,
// den.  The rule builder proposes (num, den) and accepts it only after the
// GPU has compared this very function with the double-precision table entry
// by entry; otherwise the table is used.  See ClosedForm in fqnm_internal.h.
#pragma once

#include "fqnm_internal.h"

namespace fqnm {

__device__ __forceinline__ int cf_eval(int q, const ClosedForm& c)
{
    const uint32_t x = (uint32_t)(q - c.base);
    const uint32_t t = x * c.num;
    const uint32_t d = (uint32_t)(((unsigned long long)t * c.magic) >> c.shift);
    const uint32_t r = t - d * c.den;
    uint32_t up;
    if (c.rounding == FQNM_ROUND_HALF_EVEN) {
        // tie goes to the even neighbour: d keeps the parity of floor(v)
        // because c0 is even
        up = (2u * r + (d & 1u)) > c.den;
    } else if (c.rounding == FQNM_ROUND_HALF_AWAY) {
        up = (2u * r > c.den) || (2u * r == c.den && q >= 0);
    } else {
        up = 0u;
    }
    return (int)(d + up) + c.c0;
}

}  // namespace fqnm
