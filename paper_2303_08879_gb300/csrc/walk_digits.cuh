// walk_digits.cuh -- the exact digit products of the tensor-core engine,
// shared by the all-detected walk (walk_diag_impl.cuh) and the conditional
// walk (walk_cond.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fk {

constexpr int kNDig = 7;                                    // base-256 digits per value
constexpr unsigned long long kMagicBits = 0x4B400000ull;   // bit pattern of the fp32 1.5 * 2^23

// A real product sum_c R[r][c] x[c] is computed exactly on the fp16 tensor
// cores (an Ozaki-type split): each value is turned into a 56-bit fixed
// point integer relative to a power of two shared along the contraction
// (per row r of R, per pivot for x), written as seven balanced base-256
// digits in [-128, 127] (exact in fp16), and the digit products are summed
// in fp32 per digit diagonal d = s + u <= 6.  Every partial sum is an
// integer below 2^22 in magnitude (|digit product| <= 2^14, at most 7 x 32
// terms), so fp32 holds it exactly; the diagonals are recombined in int64
// and scaled back by an exponent shift.  Dropped diagonals and the
// fixed-point cut leave a relative error near 2^-53 of the largest term,
// like FP64.

__device__ __forceinline__ int fexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// 2^e as a double for e in [-1022, 1023].
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// v 2^k for v = 0 or an integer-valued double: the exponent field moves by
// k while the result stays normal (exact, no floating-point instruction);
// otherwise two power-of-two factors, the first exact, so a subnormal or
// infinite result is rounded once.
__device__ __forceinline__ double scale2(double v, int k)
{
    const long long bits = __double_as_longlong(v);
    const int f = (int)((bits >> 52) & 0x7ff);
    if (f == 0) return v;   // zero
    if (f + k >= 1 && f + k <= 2046) return __longlong_as_double(bits + ((long long)k << 52));
    k = max(k, -2044);   // |v| < 2^64: anything smaller is zero after rounding anyway
    const int k1 = k / 2;
    return v * pow2(k1) * pow2(k - k1);
}

// Biased fixed point U = round(v * 2^(1076 - fmax)) + 0x0080808080808080:
// |round(...)| < 2^54, so 0 < U < 2^56 and byte k of U minus 128 is the
// k-th balanced base-256 digit.  fmax < 26 (values below 2^-997) gives 0.
// With ND < 7 digits the point moves 8 (7 - ND) bits up (|round| <
// 2^(8 ND - 2)) and the bias keeps ND bytes of 0x80.
template <int ND = kNDig>
__device__ __forceinline__ uint64_t to_fixed(double v, int fmax)
{
    constexpr int sh = 8 * (kNDig - ND);
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int f = (hi >> 20) & 0x7ff;
    long long X = 0;
    if (f != 0 && fmax >= 26) {
        const unsigned long long m =
            ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
        const int q = min(fmax - f + sh, 63);
        X = (long long)((((m << 2) >> q) + 1ull) >> 1);
        if (hi >> 31) X = -X;
    }
    return (uint64_t)(X + (0x0080808080808080ll >> sh));
}

// The seven digits of a pair (lo, hi) of biased fixed points as packed
// fp16 words: word s = digit s (0 = most significant) of lo in bits 0-15,
// of hi in bits 16-31.  Bytes k of lo and hi are first interleaved, then
// one byte permute places each as the low mantissa byte of an fp16 with
// exponent field 25 (the value 1024 + byte), and one packed fp16
// subtraction of 1152 leaves byte - 128, the balanced digit, exactly.
template <int ND = kNDig>
__device__ __forceinline__ void digit_words(uint64_t lo, uint64_t hi, uint32_t (&w)[ND])
{
    const uint32_t l0 = (uint32_t)lo, l1 = (uint32_t)(lo >> 32);
    const uint32_t h0 = (uint32_t)hi, h1 = (uint32_t)(hi >> 32);
    // t[k >> 1]: byte k of lo at byte 2 (k & 1), of hi at byte 2 (k & 1) + 1
    const uint32_t t[4] = {__byte_perm(l0, h0, 0x5140), __byte_perm(l0, h0, 0x7362),
                           __byte_perm(l1, h1, 0x5140), __byte_perm(l1, h1, 0x7362)};
#pragma unroll
    for (int sl = 0; sl < ND; ++sl) {
        const int k = ND - 1 - sl;
        const uint32_t v = __byte_perm(t[k >> 1], 0x64646464u, (k & 1) ? 0x4342 : 0x4140);
        uint32_t d;
        asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(v), "r"(0x64806480u));
        w[sl] = d;
    }
}

__device__ __forceinline__ void mma_f16(float *c, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Digit diagonals d = 0..6 of one accumulator element recombined:
// sum_d acc_d 256^(5 - d), the last diagonal shifted down (floor).  For
// |acc_d| < 2^22 the fp32 sum acc_d + 1.5 * 2^23 is exact and its bit
// pattern is 0x4B400000 + acc_d, so the integers come from one add each;
// the constant those offsets contribute is removed at the end (modulo
// 2^64, where the true sum fits).
template <int ND = kNDig>
__host__ __device__ constexpr unsigned long long combine_bias()
{
    unsigned long long y = kMagicBits;
    for (int d = 1; d < ND - 1; ++d) y = (y << 8) + kMagicBits;
    return y + (kMagicBits >> 8);
}

// ND diagonals (ND = 7 above; 6 for the partial sums), each below 2^22:
// sum_d acc_d 256^(ND - 2 - d), the last one floored.
template <int ND = kNDig>
__device__ __forceinline__ long long combine_digits(const float (&acc)[ND][4], int q)
{
    unsigned long long Y = __float_as_uint(acc[0][q] + 12582912.0f);
#pragma unroll
    for (int d = 1; d < ND - 1; ++d) Y = (Y << 8) + __float_as_uint(acc[d][q] + 12582912.0f);
    Y += __float_as_uint(acc[ND - 1][q] + 12582912.0f) >> 8;
    constexpr unsigned long long bias = combine_bias<ND>();
    return (long long)(Y - bias);
}

// The same for partial sums below 2^23 in magnitude (conversions to int),
// for ND diagonals: sum_d acc_d 256^(ND - 2 - d), the last one floored.
template <int ND = kNDig>
__device__ __forceinline__ long long combine_digits_wide(const float (&acc)[ND][4], int q)
{
    long long Y = __float2int_rn(acc[0][q]);
#pragma unroll
    for (int d = 1; d < ND - 1; ++d) Y = Y * 256 + __float2int_rn(acc[d][q]);
    return Y + (long long)(__float2int_rn(acc[ND - 1][q]) >> 8);
}

// Biased fixed point of v relative to exponent field fm >= field(v)
// (no flush: the caller checks the scale), ND digits as in to_fixed.
template <int ND = kNDig>
__device__ __forceinline__ uint64_t to_fixed_rel(double v, int fm)
{
    constexpr int sh = 8 * (kNDig - ND);
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int f = (hi >> 20) & 0x7ff;
    long long X = 0;
    if (f != 0) {
        const unsigned long long m =
            ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
        const int q = min(max(fm - f, 0) + sh, 63);
        X = (long long)((((m << 2) >> q) + 1ull) >> 1);
        if (hi >> 31) X = -X;
    }
    return (uint64_t)(X + (0x0080808080808080ll >> sh));
}

}  // namespace fk
