/* opcount.cpp -- op-counting build of the oracle.  Test infrastructure, like the oracle itself:
 * only the tests and the benchmark's roofline bookkeeping use it.
 *
 * rhd_oracle.c is compiled unchanged as C++ with the keyword `double` replaced by `counted`, a
 * value type holding one double that performs every floating-point operation exactly as a double
 * does and counts it.  The oracle's arithmetic, its order and its control flow are untouched, so
 * the counts are those of the plain FP64 reference algorithm (its loops, its halo work, its
 * branches on the data).  `counted` has the size and alignment of a double, so the exported
 * orc_* functions keep the oracle's C ABI and take the same arrays and parameter struct.
 *
 * Counted classes: add (additions and subtractions), mul, div, sqrt, cmp (comparisons, which
 * include every min / max / clamp written as a comparison), abs.  Negation and conversions to or
 * from integers are free.  Single-threaded (the counters are plain globals).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

namespace opc {
struct Counts {
    unsigned long long add, mul, div, sqrt, cmp, abs;
};
static Counts g_counts;
}  // namespace opc

struct counted {
    double v;
    counted() = default;
    counted(double x) : v(x) {}
    template <class T, typename std::enable_if<std::is_integral<T>::value, int>::type = 0>
    counted(T x) : v((double)x) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    explicit operator long long() const { return (long long)v; }
    counted operator-() const { return counted(-v); }
    counted operator+() const { return *this; }
    counted& operator+=(counted o) { ++opc::g_counts.add; v += o.v; return *this; }
    counted& operator-=(counted o) { ++opc::g_counts.add; v -= o.v; return *this; }
    counted& operator*=(counted o) { ++opc::g_counts.mul; v *= o.v; return *this; }
    counted& operator/=(counted o) { ++opc::g_counts.div; v /= o.v; return *this; }
};
static_assert(sizeof(counted) == sizeof(double) && alignof(counted) == alignof(double), "layout of double");
static_assert(std::is_trivially_copyable<counted>::value, "plain value");

inline counted operator+(counted a, counted b) { ++opc::g_counts.add; return counted(a.v + b.v); }
inline counted operator-(counted a, counted b) { ++opc::g_counts.add; return counted(a.v - b.v); }
inline counted operator*(counted a, counted b) { ++opc::g_counts.mul; return counted(a.v * b.v); }
inline counted operator/(counted a, counted b) { ++opc::g_counts.div; return counted(a.v / b.v); }
inline bool operator<(counted a, counted b) { ++opc::g_counts.cmp; return a.v < b.v; }
inline bool operator>(counted a, counted b) { ++opc::g_counts.cmp; return a.v > b.v; }
inline bool operator<=(counted a, counted b) { ++opc::g_counts.cmp; return a.v <= b.v; }
inline bool operator>=(counted a, counted b) { ++opc::g_counts.cmp; return a.v >= b.v; }
inline bool operator==(counted a, counted b) { ++opc::g_counts.cmp; return a.v == b.v; }
inline bool operator!=(counted a, counted b) { ++opc::g_counts.cmp; return a.v != b.v; }
inline counted sqrt(counted a) { ++opc::g_counts.sqrt; return counted(::sqrt(a.v)); }
inline counted fabs(counted a) { ++opc::g_counts.abs; return counted(::fabs(a.v)); }
inline bool isfinite(counted a) { return std::isfinite(a.v); }

#define double counted
#include "rhd_oracle.c"
#undef double

extern "C" {
/* Zero the counters and run the oracle's loops on one thread. */
void opc_reset(void)
{
    memset(&opc::g_counts, 0, sizeof(opc::g_counts));
    omp_set_num_threads(1);
}
/* out[6] = add, mul, div, sqrt, cmp, abs since the last opc_reset. */
void opc_counts(unsigned long long out[6])
{
    out[0] = opc::g_counts.add;
    out[1] = opc::g_counts.mul;
    out[2] = opc::g_counts.div;
    out[3] = opc::g_counts.sqrt;
    out[4] = opc::g_counts.cmp;
    out[5] = opc::g_counts.abs;
}
}
