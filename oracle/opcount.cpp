/*
 * opcount.cpp -- operation-counting build of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE, like the oracle itself. rmhd_oracle.c is compiled here
 * unchanged as C++, with its scalar type `double` replaced by `counted`, a
 * one-double wrapper whose +, -, x, / and sqrt add one to a global counter
 * each and then do exactly the FP64 operation (so every result is bitwise
 * that of the plain build, which a test checks).
 *
 * Not counted: negation, fabs, fmax, floor, ldexp and comparisons; operations
 * whose operands are all literal constants (they stay plain double arithmetic,
 * folded by the compiler); and trivial operations with an identity operand --
 * a product with an exact 0, +1 or -1, a quotient by +-1 or of 0, a sum or
 * difference with an exact 0. The oracle writes every cross product and the
 * B and E fluxes as full sums over the Levi-Civita symbol (27 products for a
 * cross product) so that they can be checked by eye; the rule counts only
 * the terms that do arithmetic (a cross product: 6 products and 3
 * differences). On data without exact zeros or unit values, which is what the
 * counts are taken on, every remaining operation is one the method needs.
 *
 * Single-threaded (built without OpenMP): the counters are plain globals.
 * orc_count_reset() zeroes them; orc_count_get(out) writes (add, sub, mul,
 * div, sqrt).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#include <cmath>

namespace {
long long g_ops[5];
}

struct counted {
    double v;
    counted() = default;
    counted(double d) : v(d) {}
    explicit operator double() const { return v; }
};

inline bool unit(double x) { return x == 1.0 || x == -1.0; }
inline counted operator+(counted a, counted b) {
    if (a.v != 0.0 && b.v != 0.0) ++g_ops[0];
    return counted(a.v + b.v);
}
inline counted operator-(counted a, counted b) {
    if (a.v != 0.0 && b.v != 0.0) ++g_ops[1];
    return counted(a.v - b.v);
}
inline counted operator*(counted a, counted b) {
    if (a.v != 0.0 && b.v != 0.0 && !unit(a.v) && !unit(b.v)) ++g_ops[2];
    return counted(a.v * b.v);
}
inline counted operator/(counted a, counted b) {
    if (a.v != 0.0 && !unit(b.v)) ++g_ops[3];
    return counted(a.v / b.v);
}
inline counted operator-(counted a) { return counted(-a.v); }
inline counted &operator+=(counted &a, counted b) { a = a + b; return a; }
inline counted &operator-=(counted &a, counted b) { a = a - b; return a; }
inline counted &operator*=(counted &a, counted b) { a = a * b; return a; }
inline counted &operator/=(counted &a, counted b) { a = a / b; return a; }
inline bool operator<(counted a, counted b) { return a.v < b.v; }
inline bool operator>(counted a, counted b) { return a.v > b.v; }
inline bool operator<=(counted a, counted b) { return a.v <= b.v; }
inline bool operator>=(counted a, counted b) { return a.v >= b.v; }
inline bool operator==(counted a, counted b) { return a.v == b.v; }
inline bool operator!=(counted a, counted b) { return a.v != b.v; }
inline counted sqrt(counted a) { ++g_ops[4]; return counted(std::sqrt(a.v)); }
inline counted fabs(counted a) { return counted(std::fabs(a.v)); }
inline counted fmax(counted a, counted b) { return counted(std::fmax(a.v, b.v)); }
inline counted floor(counted a) { return counted(std::floor(a.v)); }
inline counted ldexp(counted a, int e) { return counted(std::ldexp(a.v, e)); }
inline bool isfinite(counted a) { return std::isfinite(a.v); }

#define double counted
extern "C" {
#include "rmhd_oracle.c"
}
#undef double

extern "C" void orc_count_reset(void) { for (int k = 0; k < 5; ++k) g_ops[k] = 0; }
extern "C" void orc_count_get(long long *out) { for (int k = 0; k < 5; ++k) out[k] = g_ops[k]; }
