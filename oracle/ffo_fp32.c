/* ffo_fp32.c -- the oracle's formulas evaluated in single precision.
 *
 * TEST INFRASTRUCTURE ONLY, and not a parity reference.  This unit compiles
 * ffo.c once more with every `double` turned into `float` (the C library's
 * elementary functions stay the double-precision ones, so exp, expm1 and the
 * like come back rounded once to float).  The result is an FP32 computation of
 * exactly the oracle's right-hand sides and RK4 / Euler steps, in the oracle's
 * order, with no contraction and correctly rounded exponentials.
 *
 * The tests use its error against the FP64 oracle as a yardstick: how close
 * any FP32 evaluation of the same formulas can come to the FP64 result over a
 * given horizon.  Only ffo_integrate is meant to be called (its arguments are
 * all pointers and integers, so the FP64 wrapper's signature serves it with
 * float32 arrays).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define double float
#include "ffo.c"
