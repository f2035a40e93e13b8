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

} // namespace nls
