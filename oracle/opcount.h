/*
 * opcount.h -- an operation-counting scalar for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY (like the rest of oracle/).  Compiling the oracle's
 * sources as C++ with `real` = or_creal runs the same code while counting every
 * floating-point operation of the plain formulation: add/sub, mul, div, sqrt,
 * transcendentals (sin, cos, exp) and comparisons, in or_ops.  The counts measure
 * the oracle's own arithmetic; they never enter a parity check.
 */
#ifndef MPPI_ORACLE_OPCOUNT_H
#define MPPI_ORACLE_OPCOUNT_H
#ifdef __cplusplus
#include <cmath>

struct or_opcounts {
    unsigned long long add, mul, div, sqrt, trans, cmp;
};
inline or_opcounts or_ops = {0, 0, 0, 0, 0, 0};

struct or_creal {
    double v;
    or_creal() = default;
    or_creal(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator float() const { return (float)v; }
    explicit operator int() const { return (int)v; }
    or_creal& operator+=(or_creal o) { or_ops.add++; v += o.v; return *this; }
    or_creal& operator-=(or_creal o) { or_ops.add++; v -= o.v; return *this; }
    or_creal& operator*=(or_creal o) { or_ops.mul++; v *= o.v; return *this; }
    or_creal& operator/=(or_creal o) { or_ops.div++; v /= o.v; return *this; }
};
inline or_creal operator+(or_creal a, or_creal b) { or_ops.add++; return or_creal(a.v + b.v); }
inline or_creal operator-(or_creal a, or_creal b) { or_ops.add++; return or_creal(a.v - b.v); }
inline or_creal operator*(or_creal a, or_creal b) { or_ops.mul++; return or_creal(a.v * b.v); }
inline or_creal operator/(or_creal a, or_creal b) { or_ops.div++; return or_creal(a.v / b.v); }
inline or_creal operator-(or_creal a) { return or_creal(-a.v); }
inline or_creal operator+(or_creal a) { return a; }
inline bool operator<(or_creal a, or_creal b) { or_ops.cmp++; return a.v < b.v; }
inline bool operator>(or_creal a, or_creal b) { or_ops.cmp++; return a.v > b.v; }
inline bool operator<=(or_creal a, or_creal b) { or_ops.cmp++; return a.v <= b.v; }
inline bool operator>=(or_creal a, or_creal b) { or_ops.cmp++; return a.v >= b.v; }
inline bool operator==(or_creal a, or_creal b) { or_ops.cmp++; return a.v == b.v; }
inline bool operator!=(or_creal a, or_creal b) { or_ops.cmp++; return a.v != b.v; }
inline or_creal sqrt(or_creal a) { or_ops.sqrt++; return or_creal(std::sqrt(a.v)); }
inline or_creal sin(or_creal a) { or_ops.trans++; return or_creal(std::sin(a.v)); }
inline or_creal cos(or_creal a) { or_ops.trans++; return or_creal(std::cos(a.v)); }
inline or_creal exp(or_creal a) { or_ops.trans++; return or_creal(std::exp(a.v)); }
inline or_creal fabs(or_creal a) { or_ops.cmp++; return or_creal(std::fabs(a.v)); }
inline or_creal floor(or_creal a) { or_ops.cmp++; return or_creal(std::floor(a.v)); }
inline or_creal fmax(or_creal a, or_creal b) { or_ops.cmp++; return or_creal(std::fmax(a.v, b.v)); }
inline or_creal fmin(or_creal a, or_creal b) { or_ops.cmp++; return or_creal(std::fmin(a.v, b.v)); }
inline bool isfinite(or_creal a) { return std::isfinite(a.v); }

extern "C" {
/* read and clear the counters: out = {add, mul, div, sqrt, trans, cmp} */
void or_opcount_take(unsigned long long out[6]);
}
#endif
#endif
