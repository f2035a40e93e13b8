// nls_dual.cuh -- forward-mode dual numbers held in registers.
//
// A Dual<N, M, T> carries a value v and the partial derivatives d[k] with
// respect to the N seeded inputs (Sec. 2.4: forward mode fills the Jacobian
// one column per seed; all N seeds are propagated in one pass).  The mask M
// records, at compile time, which partials can be non-zero: a seed u_j has
// only bit j set, sums and products take the union.  Partials outside the
// mask are never stored or computed, so the structurally-zero columns of a
// row cost nothing -- the compile-time counterpart of the sparsity-aware
// forward mode of Sec. 2.4.  Every partial that is computed is exactly the
// one a dense dual pass computes (the skipped ones are the 0 * x terms).
//
// All loops run over compile-time k, so after unrolling the mask tests fold
// away and only the live partials remain in registers.
#pragma once

#include <cstdint>

namespace nls {

#define NLS_DI __device__ __forceinline__

template <int N, uint32_t M, class T>
struct Dual {
    T v;
    T d[N];
};

template <uint32_t M>
NLS_DI constexpr bool mask_has(int k) { return (M >> k) & 1u; }

// u_J seeded with partial 1 in slot J.
template <int N, int J, class T>
NLS_DI Dual<N, (1u << J), T> seed(T v)
{
    Dual<N, (1u << J), T> r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (k == J) ? T(1) : T(0);
    return r;
}

template <int N, uint32_t A, uint32_t B, class T>
NLS_DI Dual<N, A | B, T> operator+(const Dual<N, A, T> &x, const Dual<N, B, T> &y)
{
    Dual<N, A | B, T> r;
    r.v = x.v + y.v;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (mask_has<A>(k) && mask_has<B>(k)) r.d[k] = x.d[k] + y.d[k];
        else if (mask_has<A>(k)) r.d[k] = x.d[k];
        else if (mask_has<B>(k)) r.d[k] = y.d[k];
        else r.d[k] = T(0);
    }
    return r;
}

template <int N, uint32_t A, uint32_t B, class T>
NLS_DI Dual<N, A | B, T> operator-(const Dual<N, A, T> &x, const Dual<N, B, T> &y)
{
    Dual<N, A | B, T> r;
    r.v = x.v - y.v;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (mask_has<A>(k) && mask_has<B>(k)) r.d[k] = x.d[k] - y.d[k];
        else if (mask_has<A>(k)) r.d[k] = x.d[k];
        else if (mask_has<B>(k)) r.d[k] = -y.d[k];
        else r.d[k] = T(0);
    }
    return r;
}

// product rule: (x y)' = x' y + x y'
template <int N, uint32_t A, uint32_t B, class T>
NLS_DI Dual<N, A | B, T> operator*(const Dual<N, A, T> &x, const Dual<N, B, T> &y)
{
    Dual<N, A | B, T> r;
    r.v = x.v * y.v;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (mask_has<A>(k) && mask_has<B>(k)) r.d[k] = x.d[k] * y.v + x.v * y.d[k];
        else if (mask_has<A>(k)) r.d[k] = x.d[k] * y.v;
        else if (mask_has<B>(k)) r.d[k] = x.v * y.d[k];
        else r.d[k] = T(0);
    }
    return r;
}

template <int N, uint32_t A, class T>
NLS_DI Dual<N, A, T> operator*(T c, const Dual<N, A, T> &x)
{
    Dual<N, A, T> r;
    r.v = c * x.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = mask_has<A>(k) ? c * x.d[k] : T(0);
    return r;
}

template <int N, uint32_t A, class T>
NLS_DI Dual<N, A, T> operator+(const Dual<N, A, T> &x, T c)
{
    Dual<N, A, T> r = x;
    r.v = x.v + c;
    return r;
}

template <int N, uint32_t A, class T>
NLS_DI Dual<N, A, T> operator-(const Dual<N, A, T> &x, T c)
{
    Dual<N, A, T> r = x;
    r.v = x.v - c;
    return r;
}

template <int N, uint32_t A, class T>
NLS_DI Dual<N, A, T> operator-(T c, const Dual<N, A, T> &x)
{
    Dual<N, A, T> r;
    r.v = c - x.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = mask_has<A>(k) ? -x.d[k] : T(0);
    return r;
}

// x^3.  Plain numbers and jets take x * x * x; a dual takes its partials as
// 3 x^2 dx (two multiplies once dx is a seed's 1) rather than through the
// product rule twice.
template <class X>
NLS_DI auto cube(const X &x)
{
    return x * x * x;
}
template <int N, uint32_t A, class T>
NLS_DI Dual<N, A, T> cube(const Dual<N, A, T> &x)
{
    Dual<N, A, T> r;
    const T x2 = x.v * x.v;
    const T s = T(3) * x2;
    r.v = x2 * x.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = mask_has<A>(k) ? s * x.d[k] : T(0);
    return r;
}

NLS_DI double nls_exp(double x) { return ::exp(x); }
NLS_DI float nls_exp(float x) { return ::expf(x); }

// (e^x)' = e^x x'
template <int N, uint32_t A, class T>
NLS_DI Dual<N, A, T> exp(const Dual<N, A, T> &x)
{
    Dual<N, A, T> r;
    r.v = nls_exp(x.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = mask_has<A>(k) ? r.v * x.d[k] : T(0);
    return r;
}

NLS_DI double exp(double x) { return nls_exp(x); }
NLS_DI float exp(float x) { return nls_exp(x); }

// ---------------------------------------------------------------------------
// Second-order Taylor numbers along one direction a: evaluated on
// x(t) = u + t a, a Jet carries x(0), x'(0) and x''(0), so a residual row
// evaluated on jets yields d^2/dt^2 F_i(u + t a) at t = 0 = (H a a)_i, the
// term Halley's method (Sec. 2.1, Eq. 3) needs, by forward mode and without
// forming the n x n x n second derivative.  S2 = false marks, at compile
// time, a jet whose second derivative is structurally zero (the seeds and
// everything linear in them), so linear parts of a residual cost two
// operations per term instead of three.
template <class T, bool S2>
struct Jet {
    T v, d1, d2;
};

template <class T, bool A, bool B>
NLS_DI Jet<T, A || B> operator+(const Jet<T, A> &x, const Jet<T, B> &y)
{
    Jet<T, A || B> r;
    r.v = x.v + y.v;
    r.d1 = x.d1 + y.d1;
    if constexpr (A && B) r.d2 = x.d2 + y.d2;
    else if constexpr (A) r.d2 = x.d2;
    else if constexpr (B) r.d2 = y.d2;
    else r.d2 = T(0);
    return r;
}

template <class T, bool A, bool B>
NLS_DI Jet<T, A || B> operator-(const Jet<T, A> &x, const Jet<T, B> &y)
{
    Jet<T, A || B> r;
    r.v = x.v - y.v;
    r.d1 = x.d1 - y.d1;
    if constexpr (A && B) r.d2 = x.d2 - y.d2;
    else if constexpr (A) r.d2 = x.d2;
    else if constexpr (B) r.d2 = -y.d2;
    else r.d2 = T(0);
    return r;
}

// (x y)'' = x'' y + 2 x' y' + x y''
template <class T, bool A, bool B>
NLS_DI Jet<T, true> operator*(const Jet<T, A> &x, const Jet<T, B> &y)
{
    Jet<T, true> r;
    r.v = x.v * y.v;
    r.d1 = x.d1 * y.v + x.v * y.d1;
    T s = T(2) * x.d1 * y.d1;
    if constexpr (A) s = s + x.d2 * y.v;
    if constexpr (B) s = s + x.v * y.d2;
    r.d2 = s;
    return r;
}

template <class T, bool A>
NLS_DI Jet<T, A> operator*(T c, const Jet<T, A> &x)
{
    Jet<T, A> r;
    r.v = c * x.v;
    r.d1 = c * x.d1;
    r.d2 = A ? c * x.d2 : T(0);
    return r;
}

template <class T, bool A>
NLS_DI Jet<T, A> operator+(const Jet<T, A> &x, T c)
{
    Jet<T, A> r = x;
    r.v = x.v + c;
    return r;
}

template <class T, bool A>
NLS_DI Jet<T, A> operator-(const Jet<T, A> &x, T c)
{
    Jet<T, A> r = x;
    r.v = x.v - c;
    return r;
}

template <class T, bool A>
NLS_DI Jet<T, A> operator-(T c, const Jet<T, A> &x)
{
    Jet<T, A> r;
    r.v = c - x.v;
    r.d1 = -x.d1;
    r.d2 = A ? -x.d2 : T(0);
    return r;
}

// (e^x)'' = e^x (x'^2 + x'')
template <class T, bool A>
NLS_DI Jet<T, true> exp(const Jet<T, A> &x)
{
    Jet<T, true> r;
    r.v = nls_exp(x.v);
    r.d1 = r.v * x.d1;
    T s = x.d1 * x.d1;
    if constexpr (A) s = s + x.d2;
    r.d2 = r.v * s;
    return r;
}

} // namespace nls
