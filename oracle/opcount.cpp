/*
 * Operation-counting build of the FP64 CPU oracle (es_oracle.c).
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE: it counts the floating-point operations the
 * oracle performs, i.e. the method's arithmetic in the order and form the paper writes
 * it (the two-point flux of every pair of every interface formed from scratch, the
 * eigenvector matrices written out, and so on).  The benchmark divides these counts,
 * per interface and per node, by the measured kernel times to state the algorithmic
 * flop rate of the CUDA kernels.  Nothing of the CUDA library is compiled or linked here.
 *
 * The oracle source is compiled as C++ with `double` replaced by cdouble, a standard
 * layout wrapper of one binary64 value whose operators do exactly the binary64
 * operation and count it.  The results are therefore bit for bit those of the plain
 * oracle (both builds use -ffp-contract=off); the same C entry points are exported,
 * plus or_op_reset / or_op_read.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct OpCounts {
    long long add;     /* additions and subtractions */
    long long mul;     /* multiplications */
    long long div;     /* divisions */
    long long sqrt;    /* square roots */
    long long log;     /* natural and decimal logarithms */
    long long exp;     /* exponentials and powers */
    long long cmp;     /* comparisons, fabs (no arithmetic result) */
};

static OpCounts g_ops;

struct cdouble {
    double v;
    cdouble() = default;
    cdouble(double x) : v(x) {}
    explicit operator double() const { return v; }
    cdouble& operator+=(cdouble b) { ++g_ops.add; v = v + b.v; return *this; }
    cdouble& operator-=(cdouble b) { ++g_ops.add; v = v - b.v; return *this; }
    cdouble& operator*=(cdouble b) { ++g_ops.mul; v = v * b.v; return *this; }
    cdouble& operator/=(cdouble b) { ++g_ops.div; v = v / b.v; return *this; }
};

static inline cdouble operator+(cdouble a, cdouble b) { ++g_ops.add; return cdouble(a.v + b.v); }
static inline cdouble operator-(cdouble a, cdouble b) { ++g_ops.add; return cdouble(a.v - b.v); }
static inline cdouble operator*(cdouble a, cdouble b) { ++g_ops.mul; return cdouble(a.v * b.v); }
static inline cdouble operator/(cdouble a, cdouble b) { ++g_ops.div; return cdouble(a.v / b.v); }
static inline cdouble operator-(cdouble a) { return cdouble(-a.v); }
static inline cdouble operator+(cdouble a) { return a; }
static inline bool operator<(cdouble a, cdouble b) { ++g_ops.cmp; return a.v < b.v; }
static inline bool operator>(cdouble a, cdouble b) { ++g_ops.cmp; return a.v > b.v; }
static inline bool operator<=(cdouble a, cdouble b) { ++g_ops.cmp; return a.v <= b.v; }
static inline bool operator>=(cdouble a, cdouble b) { ++g_ops.cmp; return a.v >= b.v; }
static inline bool operator==(cdouble a, cdouble b) { ++g_ops.cmp; return a.v == b.v; }
static inline bool operator!=(cdouble a, cdouble b) { ++g_ops.cmp; return a.v != b.v; }
static inline cdouble sqrt(cdouble a) { ++g_ops.sqrt; return cdouble(::sqrt(a.v)); }
static inline cdouble log(cdouble a) { ++g_ops.log; return cdouble(::log(a.v)); }
static inline cdouble log10(cdouble a) { ++g_ops.log; return cdouble(::log10(a.v)); }
static inline cdouble exp(cdouble a) { ++g_ops.exp; return cdouble(::exp(a.v)); }
static inline cdouble pow(cdouble a, cdouble b) { ++g_ops.exp; return cdouble(::pow(a.v, b.v)); }
static inline cdouble fabs(cdouble a) { ++g_ops.cmp; return cdouble(::fabs(a.v)); }

#define double cdouble
#include "es_oracle.c"
#undef double

extern "C" {

void or_op_reset(void) { memset(&g_ops, 0, sizeof(g_ops)); }

/* out[7] = {add, mul, div, sqrt, log, exp, cmp} since the last reset */
void or_op_read(long long* out)
{
    out[0] = g_ops.add;
    out[1] = g_ops.mul;
    out[2] = g_ops.div;
    out[3] = g_ops.sqrt;
    out[4] = g_ops.log;
    out[5] = g_ops.exp;
    out[6] = g_ops.cmp;
}

}  /* extern "C" */
