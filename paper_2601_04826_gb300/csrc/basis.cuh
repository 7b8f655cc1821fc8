// basis.cuh -- compile-time integrals of the shifted Legendre basis.
//
// phi_k(z) = sum_j binom(k,j) binom(k+j,j) (-z)^j  (= P_k(1-2z), so phi_k(0) = 1, z = 0
// at the bed), the basis of the shallow-moment hierarchy (Sec. 2.1.1, "Basismatrices"
// with Legendre_shifted; Sec. 3.4).  The integrals that the model needs,
//   M_k = <phi_k, phi_k>,  A_ijk = <phi_i phi_j, phi_k>,  B_kjl = <phi_k', phi_j Phi_l>,
//   C_ik = <phi_i', phi_k'>,  Phi_l(z) = int_0^z phi_l,
// are evaluated here exactly in rational arithmetic by the C++ compiler, so the
// kernels see them as literal constants and every vanishing product drops out of
// the unrolled code.
#pragma once
#include <cstdint>
#include <type_traits>

namespace zoomy {

struct Rat {
    long long n, d;
};

constexpr long long ll_abs(long long a) { return a < 0 ? -a : a; }
constexpr long long ll_gcd(long long a, long long b)
{
    a = ll_abs(a);
    b = ll_abs(b);
    while (b) {
        long long t = a % b;
        a = b;
        b = t;
    }
    return a ? a : 1;
}
constexpr Rat rat(long long n, long long d = 1)
{
    long long g = ll_gcd(n, d);
    return d < 0 ? Rat{-n / g, -d / g} : Rat{n / g, d / g};
}
constexpr Rat radd(Rat a, Rat b) { return rat(a.n * b.d + b.n * a.d, a.d * b.d); }
constexpr Rat rmul(Rat a, Rat b)
{
    long long g1 = ll_gcd(a.n, b.d), g2 = ll_gcd(b.n, a.d);
    return rat((a.n / g1) * (b.n / g2), (a.d / g2) * (b.d / g1));
}
constexpr double rdbl(Rat a) { return (double)a.n / (double)a.d; }

constexpr long long binom(int n, int k)
{
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// coefficient of z^j in phi_k, phi_k' and Phi_k
constexpr Rat phi_c(int k, int j)
{
    if (j < 0 || j > k) return rat(0);
    long long c = binom(k, j) * binom(k + j, j);
    return rat((j & 1) ? -c : c);
}
constexpr Rat dphi_c(int k, int j) { return rmul(rat(j + 1), phi_c(k, j + 1)); }
constexpr Rat Phi_c(int k, int j) { return j == 0 ? rat(0) : rmul(phi_c(k, j - 1), rat(1, j)); }

constexpr Rat intM(int k)
{
    Rat s = rat(0);
    for (int a = 0; a <= k; ++a)
        for (int b = 0; b <= k; ++b) s = radd(s, rmul(rmul(phi_c(k, a), phi_c(k, b)), rat(1, a + b + 1)));
    return s;
}
constexpr Rat intA(int i, int j, int k)
{
    Rat s = rat(0);
    for (int a = 0; a <= i; ++a)
        for (int b = 0; b <= j; ++b)
            for (int c = 0; c <= k; ++c)
                s = radd(s, rmul(rmul(rmul(phi_c(i, a), phi_c(j, b)), phi_c(k, c)), rat(1, a + b + c + 1)));
    return s;
}
constexpr Rat intB(int k, int j, int l)
{
    Rat s = rat(0);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b <= j; ++b)
            for (int c = 1; c <= l + 1; ++c)
                s = radd(s, rmul(rmul(rmul(dphi_c(k, a), phi_c(j, b)), Phi_c(l, c)), rat(1, a + b + c + 1)));
    return s;
}
constexpr Rat intC(int i, int k)
{
    Rat s = rat(0);
    for (int a = 0; a < i; ++a)
        for (int b = 0; b < k; ++b) s = radd(s, rmul(rmul(dphi_c(i, a), dphi_c(k, b)), rat(1, a + b + 1)));
    return s;
}

// Model coefficients as they enter the equations (already divided by M_k).
//   flux:  (1/M_k) A_ijk                  -> fluxA(i,j,k)
//   NC:    (1/M_k) B_kjl  (j >= 1)         -> ncB(k,j,l)
//   bulk:  (1/M_k) C_ik                    -> visC(i,k)
//   bed:   phi_k(0)/M_k = 2k+1             -> bedW(k)
constexpr double fluxA(int i, int j, int k) { return rdbl(rmul(intA(i, j, k), rat(intM(k).d, intM(k).n))); }
constexpr double ncB(int k, int j, int l) { return rdbl(rmul(intB(k, j, l), rat(intM(k).d, intM(k).n))); }
constexpr double visC(int i, int k) { return rdbl(rmul(intC(i, k), rat(intM(k).d, intM(k).n))); }
constexpr double bedW(int k) { return rdbl(rmul(phi_c(k, 0), rat(intM(k).d, intM(k).n))); }

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

}  // namespace zoomy
