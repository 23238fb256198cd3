// tcgen05 building blocks shared by the exact-slice tensor-core kernels: shared-memory operand descriptors in the
// canonical no-swizzle K-major layout, the BF16 MMA with FP32 accumulation into tensor memory, commit / bounded
// mbarrier waits, tensor-memory loads, and the exact slicing of FP64 values into four BF16 digits.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace osv {

// every spin-wait on an mbarrier gives up after this many cycles (~2 s): the kernel then reports an error
constexpr long long kTcWaitBudget = 4LL << 30;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) in a no-swizzle K-major image whose K extent is kext (a multiple of 8): core
// matrices of 8 rows x 16 bytes, K-adjacent core matrices 128 B apart (LBO), 8-row groups 16 kext B apart (SBO)
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int kext) {
    return (uint32_t)((r >> 3) * (16 * kext) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, LBO 128 B, SBO sbo bytes, no swizzle (sm_100 descriptor version)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, shape M x N (M = 128; N % 16 == 0)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool neg_a = false) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void tc_mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate ? 1u : 0u));
}

// arrive on bar once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// wait for the given phase parity of bar, bounded by `budget` clock cycles (<= 0: kTcWaitBudget): false when the
// budget ran out.  Main-loop waits take the caller's budget; the tear-down waits for work already committed (MMAs
// and copies that complete on their own) always take the full kTcWaitBudget.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, long long budget = kTcWaitBudget) {
    if (budget <= 0) budget = kTcWaitBudget;
    const long long t0 = clock64();
    uint32_t done = 0;
    while (true) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes (one value per lane and column)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// (hi, lo) += x with Knuth's two-sum (exact error term; FP32 only)
__device__ __forceinline__ void two_sum_f32(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// d 2^(-8 i) for an integer |d| < 2^22 with one integer add and one FP32 subtraction, both exact: the bit pattern
// of 1.5 2^(23 - 8 i) plus d is the float 1.5 2^(23 - 8 i) + d 2^(-8 i) (its unit in the last place is 2^(-8 i)).
// Keeps the integer-to-float conversion off the reduced-rate conversion path.
template <int I>
__device__ __forceinline__ float digit_to_float(int d) {
    constexpr int kBits = 0x4B400000 - ((8 * I) << 23);   // 1.5 2^(23 - 8 I)
    return __fsub_rn(__int_as_float(kBits + d), __int_as_float(kBits));
}

// x = N 2^(e-31) + rounding (|x| <= 2^e), N cut into four signed base-256 digits; slice i returned as s_i 2^(-8 i)
// (exact BF16 values).  Inf / NaN propagate as NaN; zero and subnormal inputs slice to zero.
__device__ __forceinline__ void slice4_exact(double x, int e, float *s) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0x7FF) {
        s[0] = s[1] = s[2] = s[3] = __int_as_float(0x7FC00000);
        return;
    }
    long long n = 0;
    if (ex != 0) {
        const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;   // value = mant 2^(ex-1075)
        const int sh = 1075 - ex + e - 31;                   // N = mant / 2^sh, sh >= 21 since |x| <= 2^e
        if (sh < 63) n = (mant + (1LL << (sh - 1))) >> sh;
        if (bits < 0) n = -n;
    }
    const int s0 = (int)((n + (1LL << 23)) >> 24);
    int r = (int)(n - ((long long)s0 << 24));
    const int s1 = (r + (1 << 15)) >> 16;
    r -= s1 << 16;
    const int s2 = (r + (1 << 7)) >> 8;
    const int s3 = r - (s2 << 8);
    s[0] = digit_to_float<0>(s0);
    s[1] = digit_to_float<1>(s1);
    s[2] = digit_to_float<2>(s2);
    s[3] = digit_to_float<3>(s3);
}

// |x| as its bit pattern (integer order = numeric order for finite values): maxima on the integer ALU
__device__ __forceinline__ unsigned long long abs_bits64(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}
// e with max |x| = f 2^e, f in [0.5, 1), from the bit pattern of max |x|; 0 for zero, the smallest normal
// exponent for a subnormal maximum (which slices to zero)
__device__ __forceinline__ int scale_exp_of_bits(unsigned long long b) {
    if (b == 0ULL) return 0;
    const int ex = (int)(b >> 52);
    return ex == 0 ? -1021 : ex - 1022;
}
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

}  // namespace osv
