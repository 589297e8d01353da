// Host-side number theory for the offline precompute of hefx parameter sets.
//
// Everything the kernels need that depends only on the moduli (roots of unity, inverses,
// Shoup companions, BAT digit matrices) is computed here once per parameter set, the
// "compile time" of Sec. IV-A / IV-B, and uploaded; nothing here runs per call.
#pragma once

#include <cstdint>
#include <vector>

namespace hefx {

typedef unsigned __int128 u128;

inline uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

inline uint64_t pow_mod(uint64_t b, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    b %= m;
    for (; e; e >>= 1, b = mul_mod(b, b, m))
        if (e & 1) r = mul_mod(r, b, m);
    return r;
}

// Deterministic Miller-Rabin for 64-bit n (the first 12 prime bases suffice below 3.3e24).
inline bool is_prime(uint64_t n) {
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t p : small)
        if (n % p == 0) return n == p;
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; ++s; }
    for (uint64_t a : small) {
        uint64_t x = pow_mod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mul_mod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// Smallest g whose order mod the prime q is q-1.
inline uint64_t smallest_generator(uint64_t q) {
    std::vector<uint64_t> fac;
    uint64_t m = q - 1;
    for (uint64_t p = 2; p * p <= m; p += (p == 2 ? 1 : 2))
        if (m % p == 0) {
            fac.push_back(p);
            while (m % p == 0) m /= p;
        }
    if (m > 1) fac.push_back(m);
    for (uint64_t g = 2;; ++g) {
        bool gen = true;
        for (uint64_t f : fac)
            if (pow_mod(g, (q - 1) / f, q) == 1) { gen = false; break; }
        if (gen) return g;
    }
}

inline uint64_t inv_mod(uint64_t a, uint64_t q) { return pow_mod(a, q - 2, q); }  // q prime

// psi: a primitive 2N-th root of unity, g^((q-1)/2N) for the smallest generator g.
inline uint64_t root_2n(uint64_t q, uint64_t n) { return pow_mod(smallest_generator(q), (q - 1) / (2 * n), q); }

inline uint32_t bit_reverse(uint32_t v, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i, v >>= 1) r = (r << 1) | (v & 1);
    return r;
}

// Shoup companion floor(w * 2^32 / q) for a constant w < q.
inline uint32_t shoup(uint64_t w, uint64_t q) { return (uint32_t)(((u128)w << 32) / q); }

// -q^-1 mod 2^32 by Newton iteration (q odd).
inline uint32_t neg_inv_pow2_32(uint32_t q) {
    uint32_t x = q;  // correct to 3 bits for odd q
    for (int i = 0; i < 5; ++i) x *= 2 - q * x;
    return (uint32_t)(0u - x);
}

}  // namespace hefx
