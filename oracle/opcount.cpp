/*
 * opcount.cpp -- the counter readout of the operation-counting oracle build
 * (opcount.h).  TEST INFRASTRUCTURE ONLY.
 */
#include "opcount.h"

extern "C" void or_opcount_take(unsigned long long out[6]) {
    out[0] = or_ops.add;
    out[1] = or_ops.mul;
    out[2] = or_ops.div;
    out[3] = or_ops.sqrt;
    out[4] = or_ops.trans;
    out[5] = or_ops.cmp;
    or_ops = or_opcounts{0, 0, 0, 0, 0, 0};
}
