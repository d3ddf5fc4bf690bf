// Device code shared by the fused kernels (FP32 FFT form and tensor-core DFT
// form): packed FP32x2 complex arithmetic, small DFTs with compile-time
// twiddles, the exact 4+4-bit unpack, tensor-memory access and the two
// up-channelisation passes (Sec. 3.2) that run out of tensor memory.
#pragma once

#include "bf_internal.h"

#include <cstdint>

namespace chimebf {
namespace {

// ---------------------------------------------------------------------------
// packed FP32x2 helpers (sm_100+: FADD2 / FMUL2 / FFMA2)
// ---------------------------------------------------------------------------
struct cp {            // two complex values in SoA form
    float2 re, im;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }

__device__ __forceinline__ cp cadd(cp a, cp b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ cp csub(cp a, cp b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }
// a * (-i)
__device__ __forceinline__ cp cmul_neg_i(cp a) { return {a.im, mul2(a.re, bc(-1.f))}; }
// a * (C + i S), C and S pairs (per element of the pair)
__device__ __forceinline__ cp cmulp(cp a, float2 C, float2 S) {
    return {fma2(a.im, make_float2(-S.x, -S.y), mul2(a.re, C)), fma2(a.re, S, mul2(a.im, C))};
}
__device__ __forceinline__ cp ld_cp(const float4* p) {
    const float4 v = *p;
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st_cp(float4* p, cp a) { *p = make_float4(a.re.x, a.re.y, a.im.x, a.im.y); }

// cos(2 pi e / 32), e = 0..31, rounded from double precision.
__device__ __forceinline__ constexpr float cos32(int e) {
    constexpr float t[32] = {
        1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
        7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
        0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
        -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
        -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
        -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f,
        0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
        7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f};
    return t[e & 31];
}
__device__ __forceinline__ constexpr float sin32(int e) { return cos32(e - 8); }

// a * exp(-2 pi i e / N) for N | 32 and a compile-time e (after unrolling).
template <int N>
__device__ __forceinline__ cp twiddle(cp a, int e) {
    const int k = (e * (32 / N)) & 31;               // angle in units of 2 pi / 32
    switch (k) {
        case 0: return a;
        case 8: return cmul_neg_i(a);
        case 16: return {mul2(a.re, bc(-1.f)), mul2(a.im, bc(-1.f))};
        case 24: return {mul2(a.im, bc(-1.f)), a.re};
        default: return cmulp(a, bc(cos32(k)), bc(-sin32(k)));
    }
}

__device__ __forceinline__ void dft4(cp& a0, cp& a1, cp& a2, cp& a3) {
    const cp s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3);
    // (a1 - a3) * (-i) = (a1.im - a3.im) + i (a3.re - a1.re)
    const cp d13 = {sub2(a1.im, a3.im), sub2(a3.re, a1.re)};
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, d13);
    a3 = csub(d02, d13);
}

// Radix-2 butterfly with a twiddle, factored for fused multiply-adds: with
// w = c (1 + i t), (a, b) -> (a + w b, a - w b) as p = (1 + i t) b (two FMA)
// and a +- c p (four FMA), six operations instead of a complex product and two
// complex additions (eight).  E = e in units of 2 pi / 16, w = exp(-2 pi i E / 16);
// c = cos(2 pi E / 16), t = -tan(2 pi E / 16), rounded from double precision.
template <int E>
__device__ __forceinline__ void bfly_tw(cp& a, cp& b) {
    constexpr float kc[8] = {1.f, 9.238795325e-01f, 7.071067812e-01f, 3.826834324e-01f,
                             0.f, -3.826834324e-01f, -7.071067812e-01f, -9.238795325e-01f};
    constexpr float kt[8] = {0.f, -4.142135624e-01f, -1.0f, -2.414213562e+00f,
                             0.f, 2.414213562e+00f, 1.0f, 4.142135624e-01f};
    if constexpr (E == 0) {
        const cp y = cadd(a, b), z = csub(a, b);
        a = y;
        b = z;
    } else if constexpr (E == 4) {
        // w = -i: a - i b = (a.re + b.im, a.im - b.re)
        const cp y = {add2(a.re, b.im), sub2(a.im, b.re)};
        const cp z = {sub2(a.re, b.im), add2(a.im, b.re)};
        a = y;
        b = z;
    } else {
        const float c = kc[E], t = kt[E];
        const float2 pre = fma2(b.im, bc(-t), b.re), pim = fma2(b.re, bc(t), b.im);
        const cp y = {fma2(pre, bc(c), a.re), fma2(pim, bc(c), a.im)};
        const cp z = {fma2(pre, bc(-c), a.re), fma2(pim, bc(-c), a.im)};
        a = y;
        b = z;
    }
}

// forward DFT8 (2 x 4), natural order in and out; the last stage's twiddles
// W8^k = W16^{2k} fused into its butterflies
__device__ __forceinline__ void dft8(cp (&x)[8]) {
    dft4(x[0], x[2], x[4], x[6]);
    dft4(x[1], x[3], x[5], x[7]);
    bfly_tw<0>(x[0], x[1]);
    bfly_tw<2>(x[2], x[3]);
    bfly_tw<4>(x[4], x[5]);
    bfly_tw<6>(x[6], x[7]);
    // X[k] = x[2k], X[k + 4] = x[2k + 1]
    cp y[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        y[k1] = x[2 * k1];
        y[k1 + 4] = x[2 * k1 + 1];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = y[k];
}

// second-stage group k1 of dft16: the four inputs x[4 k1 + n2] with their
// twiddles W16^{n2 k1} folded into three factored radix-2 levels
template <int K1>
__device__ __forceinline__ void dft16_group(cp& x0, cp& x1, cp& x2, cp& x3) {
    bfly_tw<(2 * K1) & 15>(x0, x2);          // x0 + w2 x2, x0 - w2 x2
    bfly_tw<(2 * K1) & 15>(x1, x3);          // u = x1 + w2 x3, v = x1 - w2 x3
    bfly_tw<K1>(x0, x1);                     // out0 = s + w1 u, out2 = s - w1 u
    bfly_tw<(K1 + 4) & 15>(x2, x3);          // out1 = d - i w1 v, out3 = d + i w1 v
}

// forward DFT16 (4 x 4), natural order in and out
__device__ __forceinline__ void dft16(cp (&x)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    dft16_group<0>(x[0], x[1], x[2], x[3]);
    dft16_group<1>(x[4], x[5], x[6], x[7]);
    dft16_group<2>(x[8], x[9], x[10], x[11]);
    dft16_group<3>(x[12], x[13], x[14], x[15]);
    // group k1 holds (out0, out2, out1, out3) in its slots (0, 1, 2, 3); X[k1 + 4 k2] = out_k2
    cp y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        y[k1] = x[4 * k1];
        y[k1 + 8] = x[4 * k1 + 1];
        y[k1 + 4] = x[4 * k1 + 2];
        y[k1 + 12] = x[4 * k1 + 3];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// ---------------------------------------------------------------------------
// 4+4-bit unpack (Table 1) of the same byte position in two rows.  The nibble
// (already shifted by 4 q bits) sits in the mantissa of 2^23; one FFMA2 scales
// it back by 16^-q and removes 2^23 and the +8 offset -- exact throughout.
// ---------------------------------------------------------------------------
template <int Q>
__device__ __forceinline__ float2 nib2(uint32_t g0, uint32_t g1) {
    constexpr uint32_t mask = 0xFu << (4 * Q);
    constexpr float s = 1.0f / float(1u << (4 * Q));
    const float f0 = __uint_as_float((g0 & mask) | 0x4B000000u);
    const float f1 = __uint_as_float((g1 & mask) | 0x4B000000u);
    return fma2(make_float2(f0, f1), bc(s), bc(-(8388608.0f * s + 8.0f)));
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// swizzles that make the 128-bit shared accesses conflict-free
__device__ __forceinline__ int ysw(int n2, int n1) { return n2 * 16 + (n1 ^ ((n2 & 7) ^ ((n2 >> 3) << 2))); }
__device__ __forceinline__ int tsw(int r, int c) { return r * 16 + (c ^ (r & 7)); }
__device__ __forceinline__ int bsw(int L) { return L ^ ((L >> 3) & 1); }

__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" :: "r"(id) : "memory"); }

// Per-lane twiddles of the N-S FFT: exp(-2 pi i n2 (2 k1 + h) / 512), k1 = 0..15.
struct PostTw {
    float2 C[16], S[16];
};

__device__ __forceinline__ void load_post(const float2* __restrict__ tw512, int n2, int h, PostTw& pt) {
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) {
        const float2 w = tw512[(n2 * (2 * k1 + h)) & (kBins - 1)];
        pt.C[k1] = bc(w.x);
        pt.S[k1] = bc(w.y);
    }
}

// E-W weights of cylinders 1..3 for one beam (cylinder 0 is the phase origin, weight 1).
struct EwW {
    float2 R[3], I[3], NI[3];
};

__device__ __forceinline__ void load_ew(const float2* __restrict__ ew, int table, int j, EwW& w) {
#pragma unroll
    for (int c = 1; c < kCyl; ++c) {
        const float2 v = ew[(table * kEw + j) * kCyl + c];
        w.R[c - 1] = bc(v.x);
        w.I[c - 1] = bc(v.y);
        w.NI[c - 1] = bc(-v.y);
    }
}

// E-W weights of beam j for frame F of a segment: the per-frame table of a
// tracking request, else the channel's static table.
__device__ __forceinline__ void load_ew_frame(const Seg& sg, const float2* __restrict__ ew, int F, int j, EwW& w) {
    if (sg.ew_frames) {
        load_ew(sg.ew_frames, F, j, w);
    } else {
        load_ew(ew, sg.table, j, w);
    }
}

__device__ __forceinline__ void load_row(const uint8_t* p, int lane, uint4 (&in)[kCyl]) {
#pragma unroll
    for (int c = 0; c < kCyl; ++c)
        in[c] = __ldg(reinterpret_cast<const uint4*>(p + c * (kFeed * kPol) + 16 * lane));
}

// ---------------------------------------------------------------------------
// tensor-memory access (tcgen05), one warp per 32-lane quarter
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_st4(uint32_t taddr, float a, float b, float c, float d) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                 :: "r"(taddr), "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)),
                    "r"(__float_as_uint(d))
                 : "memory");
}

// 64 consecutive columns: two fine channels c, c+1 x 16 residues b, as SoA pairs
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, cp (&y)[16]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
        "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
        "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        y[b].re = make_float2(__uint_as_float(r[2 * b]), __uint_as_float(r[32 + 2 * b]));
        y[b].im = make_float2(__uint_as_float(r[2 * b + 1]), __uint_as_float(r[32 + 2 * b + 1]));
    }
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// mbarriers with bounded waits
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitNs = 2000000000ull;   // default bound on every mbarrier wait (2 s)

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of phase `parity` of an mbarrier: false once `limit`
// ns have passed without it.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned long long limit) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        if (globaltimer() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}

// Work units.  A unit is an item (F, j) with all six passes, or one half of an
// item: passes 0-2 or 3-5.  When the last (or only) round of items would leave
// at least half of the CTAs idle, each item of that round becomes two half
// units on two CTAs; the second to finish adds the two halves.  Every output is the sum of
// the two halves (H0 + H1, one addition), whether or not its item was split,
// so the result does not depend on how a request was batched.
struct Units {
    int n_full;     // items run whole: 0 .. n_full - 1
    int n_units;    // n_full + 2 x (split items)
};
__device__ __forceinline__ Units make_units(int n_items, int grid, bool can_split) {
    Units u{n_items, n_items};
    if (can_split) {
        const int rem = n_items % grid;
        if (rem > 0 && 2 * rem <= grid) {
            u.n_full = n_items - rem;
            u.n_units = u.n_full + 2 * rem;
        }
    }
    return u;
}
// item, pass range [ps0, ps1) and half (-1: whole item) of unit `un`
__device__ __forceinline__ void unit_of(const Units& u, int un, int& item, int& ps0, int& ps1, int& half) {
    if (un < u.n_full) {
        item = un;
        ps0 = 0;
        ps1 = kTds * kPol;
        half = -1;
    } else {
        const int v = un - u.n_full;
        item = u.n_full + (v >> 1);
        half = v & 1;
        ps0 = half * (kTds * kPol / 2);
        ps1 = ps0 + kTds * kPol / 2;
    }
}

// Split items: the two halves of an item run on two CTAs.  A thread publishes
// its half's partial sums, then swaps its token (launch epoch x 2 + half) into
// its slot; the thread that finds its partner's token from the same launch there
// is the second of the two and adds the halves.  Tokens of earlier launches never
// match, so an abandoned launch leaves nothing to clean up, and nothing waits.
__device__ __forceinline__ bool second_half(unsigned long long* tok, unsigned long long epoch, int half) {
    __threadfence();                                   // the published sums before the token
    const unsigned long long mine = 2ull * epoch + (unsigned long long)half;
    if (atomicExch(tok, mine) != (mine ^ 1ull)) return false;
    __threadfence();                                   // the partner's sums after its token
    return true;
}

// CTA barrier that also orders tensor-memory accesses across it.
__device__ __forceinline__ void cta_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ const uint8_t* frame_row(const Seg& sg, long long row) {
    return row < sg.carry_rows ? sg.carry + row * kInput : sg.vin + (row - sg.carry_rows) * kInput;
}

// Second up-channel pass for one thread (TMEM lane, bin half hh): 16-point DFTs
// over the residue b for fine channels q = c + 8 d, two c at a time (SoA), then
// |.|^2 into the fftshifted sub-channels (d + 8) mod 16.  With `dump` set, the
// up-channelised voltages of bin m are written instead (fine channel q' order).
__device__ __forceinline__ void upchan_pass2(uint32_t tlane, int hh, float2 (&acc)[kSub], float2* dump) {
#pragma unroll 1
    for (int cpi = 0; cpi < 4; ++cpi) {
        cp y[16];
        tmem_ld64(tlane + hh * 256 + 64 * cpi, y);
        dft16(y);
        if (dump) {
#pragma unroll
            for (int dd = 0; dd < 16; ++dd) {
                const int c0 = 2 * cpi;
                dump[(c0 + 8 * dd + kUp / 2) & (kUp - 1)] = make_float2(y[dd].re.x, y[dd].im.x);
                dump[(c0 + 1 + 8 * dd + kUp / 2) & (kUp - 1)] = make_float2(y[dd].re.y, y[dd].im.y);
            }
        } else {
#pragma unroll
            for (int dd = 0; dd < 16; ++dd) {
                const float2 p = fma2(y[dd].im, y[dd].im, mul2(y[dd].re, y[dd].re));
                acc[(dd + 8) & 15] = add2(acc[(dd + 8) & 15], p);
            }
        }
    }
}

// The same with one float per sub-channel: the two fine channels of a SoA pair
// are added before they join the running sum.
__device__ __forceinline__ void upchan_pass2(uint32_t tlane, int hh, float (&acc)[kSub], float2* dump) {
#pragma unroll 1
    for (int cpi = 0; cpi < 4; ++cpi) {
        cp y[16];
        tmem_ld64(tlane + hh * 256 + 64 * cpi, y);
        dft16(y);
        if (dump) {
#pragma unroll
            for (int dd = 0; dd < 16; ++dd) {
                const int c0 = 2 * cpi;
                dump[(c0 + 8 * dd + kUp / 2) & (kUp - 1)] = make_float2(y[dd].re.x, y[dd].im.x);
                dump[(c0 + 1 + 8 * dd + kUp / 2) & (kUp - 1)] = make_float2(y[dd].re.y, y[dd].im.y);
            }
        } else {
#pragma unroll
            for (int dd = 0; dd < 16; ++dd) {
                const float2 p = fma2(y[dd].im, y[dd].im, mul2(y[dd].re, y[dd].re));
                acc[(dd + 8) & 15] += p.x + p.y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the tensor-core forms' accumulator layout: lane = bin, columns [0, 128) = Re X(t),
// [128, 256) = Im X(t) of block time t = 16 a + b
// ---------------------------------------------------------------------------
// TMEM access for the split Re/Im layout: 16 two-column loads (Re at base +
// 16 a + b0, Im at base + 128 + 16 a + b0, a = 0..7) -> SoA pairs (b0, b0 + 1).
__device__ __forceinline__ void tmem_ld_p1(uint32_t base, cp (&z)[8]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2, %3}, [%33];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%34];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6, %7}, [%35];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8, %9}, [%36];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10, %11}, [%37];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12, %13}, [%38];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14, %15}, [%39];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%16, %17}, [%40];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%18, %19}, [%41];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%20, %21}, [%42];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%22, %23}, [%43];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%24, %25}, [%44];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%26, %27}, [%45];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%28, %29}, [%46];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%30, %31}, [%47];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(base), "r"(base + 16), "r"(base + 32), "r"(base + 48), "r"(base + 64), "r"(base + 80),
          "r"(base + 96), "r"(base + 112), "r"(base + 128), "r"(base + 144), "r"(base + 160), "r"(base + 176),
          "r"(base + 192), "r"(base + 208), "r"(base + 224), "r"(base + 240)
        : "memory");
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        z[a].re = make_float2(__uint_as_float(r[2 * a]), __uint_as_float(r[2 * a + 1]));
        z[a].im = make_float2(__uint_as_float(r[16 + 2 * a]), __uint_as_float(r[16 + 2 * a + 1]));
    }
}

__device__ __forceinline__ void tmem_st2(uint32_t taddr, float a, float b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};"
                 :: "r"(taddr), "r"(__float_as_uint(a)), "r"(__float_as_uint(b)) : "memory");
}

// 32 consecutive columns -> 32 floats
__device__ __forceinline__ void tmem_ld32f(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// First up-channel pass in place on the split layout (t = 16 a + b): 8-point
// DFT over a for the residue pair (b0, b0 + 1), twiddled by exp(-2 pi i b c / 128).
__device__ __forceinline__ void upchan_pass1_split(uint32_t base, const float4* tw_s, int sub, int nsub) {
#pragma unroll 1
    for (int bp = sub; bp < 8; bp += nsub) {
        const int b0 = 2 * bp;
        cp z[8];
        tmem_ld_p1(base + b0, z);
        dft8(z);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (c) {
                const float4 tw = tw_s[bp * 8 + c];
                z[c] = cmulp(z[c], make_float2(tw.x, tw.y), make_float2(tw.z, tw.w));
            }
            tmem_st2(base + 16 * c + b0, z[c].re.x, z[c].re.y);
            tmem_st2(base + 128 + 16 * c + b0, z[c].im.x, z[c].im.y);
        }
    }
}

// Second pass on the split layout: Re of (c, b) at 16 c + b, Im at 128 + 16 c + b.
__device__ __forceinline__ void upchan_pass2_split(uint32_t base, float2 (&acc)[kSub], float2* dump, int sub,
                                                   int nsub) {
#pragma unroll 1
    for (int cpi = sub; cpi < 4; cpi += nsub) {
        float re[32], im[32];
        tmem_ld32f(base + 32 * cpi, re);
        tmem_ld32f(base + 128 + 32 * cpi, im);
        cp y[16];
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            y[b].re = make_float2(re[b], re[16 + b]);
            y[b].im = make_float2(im[b], im[16 + b]);
        }
        dft16(y);
        if (dump) {
#pragma unroll
            for (int dd = 0; dd < 16; ++dd) {
                const int c0 = 2 * cpi;
                dump[(c0 + 8 * dd + kUp / 2) & (kUp - 1)] = make_float2(y[dd].re.x, y[dd].im.x);
                dump[(c0 + 1 + 8 * dd + kUp / 2) & (kUp - 1)] = make_float2(y[dd].re.y, y[dd].im.y);
            }
        } else {
#pragma unroll
            for (int dd = 0; dd < 16; ++dd) {
                const float2 p = fma2(y[dd].im, y[dd].im, mul2(y[dd].re, y[dd].re));
                acc[(dd + 8) & 15] = add2(acc[(dd + 8) & 15], p);
            }
        }
    }
}

}  // namespace
}  // namespace chimebf
