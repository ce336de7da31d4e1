// The walk-count SpMV of Algorithm 1, fused with the bound update:
//
//   s_r(u) = alpha * sum_{u->x} s_{r-1}(x)        (Eq. 5, scaled by alpha^r)
//   c_r(u) = c_{r-1}(u) + s_r(u)
//   l_r, u_r from c_r and s_r for u in M; u joins the candidate list when
//   l_r(u) >= theta_{r-1}.
//
// The graph is stored in internal order (katz_relabel.cu): rows grouped by
// degree class, largest first.  Rows are processed in four row modes chosen by
// degree, so the lanes that share a row (or the rows that share a warp) carry
// equal work, and no lane waits on a merge search or a block barrier:
//   THREAD  deg <= 16         one thread per row
//   OCTET   16 < deg <= 128   eight lanes per row
//   WARP    128 < deg <= 2048 one warp per row
//   CHUNK   deg > 2048        one warp per 2048-arc chunk; spmv_chunk_fixup adds
//                             a row's chunk sums as a pairwise tree and finishes it
// The walk vector is gathered with read-only loads (one L2 request per arc:
// this access, not HBM bandwidth, bounds the kernel on power-law graphs).
//
// Row sums of an FP64 level are exact: each lane adds its terms into a
// 128-bit fixed-point accumulator whose scale follows the largest exponent
// seen (XAcc below), lanes and chunks merge their accumulators, and the
// total is rounded once to FP64.  A row sum is therefore the correctly
// rounded sum of its terms (up to a truncation near 2^-90 relative), for any
// order and any split of the terms over lanes, warps or chunks: the full
// SpMV, the repair of single rows and the chunked hub rows all give the same
// bits.  The adds run on the integer pipes; GB300 executes FP64 additions at
// a small fraction of its integer rate, and one FP64 add per arc was the
// limit of the kernel.
//
// FP32 levels (FP32-certified mode) add in FP32 in a fixed order: each lane
// adds its terms eight at a time as a pairwise tree and chains the
// eight-term sums; lanes then meet in a shuffle tree.  The longest chain of
// additions in a row sum (max_sum_depth) enters that mode's rounding-error
// bound.
//
// Level types: FP64 mode computes every level in FP64.  The FP32-certified
// mode starts in FP64 and computes the levels from Ctrl::f32_from on in FP32
// (FP32 storage, FP32 sums, FP32 multiply by alpha), adding them to the
// separate partial sum c32.
#include <cooperative_groups.h>
#include <stdint.h>

#include <algorithm>

#include "katz_common.cuh"

namespace cg = cooperative_groups;

namespace katz {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLOCK = 256;
constexpr int WARPS = BLOCK / 32;

struct Epi {
    void* y;          // level r slot (double or float)
    double* c64;
    double* c32;
    double* lb;       // cert mode: monotone stored bounds
    double* ub;
    uint8_t* active;
    const int32_t* perm;
    double* cand_l;
    double* cand_u;
    int32_t* cand_id;
    int64_t cand_cap;
    Ctrl* ctrl;
    double theta_prev;
    BState bs;
    int store_only;   // dynamic repair: write s_r only (c and bounds are rebuilt afterwards)
    float* s32;       // FP32-certified mode, FP64 levels before the switch: s_r rounded to FP32 too
};

// Conversions between binary64 and binary32 for the non-negative finite walk
// values, on the integer pipes (the FP64 pipe of this GPU is narrow and the
// epilogue converts once per row).  Written from the IEEE 754 encodings:
// f64_to_f32_rn rounds to nearest, ties to even, into normal or subnormal
// binary32 (0 below half the smallest subnormal); f32_to_f64 is exact.  The
// GPU tests compare both with the hardware conversions.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)(b >> 52);  // biased exponent (the sign bit is 0)
    if (e == 0) return 0.0f;       // zero or a binary64 subnormal, far below binary32's range
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
    const int fe = e - 896;        // binary32 biased exponent (1023 - 127)
    if (fe >= 255) return __uint_as_float(0x7f800000u);
    const int sh = fe >= 1 ? 29 : 30 - fe;  // significand bits dropped: normal, or subnormal result
    if (sh > 60) return 0.0f;
    const unsigned long long r = m >> sh, rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    const unsigned long long q = r + ((rem > half || (rem == half && (r & 1ull))) ? 1ull : 0ull);
    // normal: q in [2^23, 2^24], a carry to 2^24 moves into the exponent field;
    // subnormal: q in [0, 2^23], 2^23 being the smallest normal
    const uint32_t bits = fe >= 1 ? (uint32_t)(((unsigned long long)fe << 23) + (q - (1ull << 23))) : (uint32_t)q;
    return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = b >> 23, m = b & 0x7FFFFFu;
    if (e == 0) {
        if (m == 0) return 0.0;
        const int hb = 31 - __clz(m);  // subnormal: m 2^-149 = 1.x 2^(hb - 149)
        const unsigned long long frac = ((unsigned long long)m << (52 - hb)) & 0xFFFFFFFFFFFFFull;
        return __longlong_as_double((long long)(((unsigned long long)(hb + 874) << 52) | frac));
    }
    const unsigned long long ed = e == 255 ? 0x7FFull : (unsigned long long)(e + 896);  // inf stays inf
    return __longlong_as_double((long long)((ed << 52) | ((unsigned long long)m << 29)));
}

// bounds and thresholds are non-negative doubles: they order like their bit patterns
__device__ __forceinline__ double nn_max(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ double nn_min(double a, double b) {
    return __longlong_as_double(min(__double_as_longlong(a), __double_as_longlong(b)));
}

// Finish row u of an FP64 level: s = alpha * sum, c64 += s, bounds, candidate.
// Finish row u of an FP32 level: s = fl32(alpha_f * sum), c32 += s, bounds, candidate.
// Candidates carry the original id.
// ZeroRows: rows without walks so far (sum and c both +0) skip the FP64
// arithmetic; alpha * +0 and +0 + +0 are +0 in every rounding mode, so the
// bits are those of the full computation.  Worth it where the FP64 pipe
// (narrow on this GPU) bounds the pass, as in the degree pass over an R-MAT
// graph whose rows are mostly isolated nodes; the gather levels, bound by
// their loads, run the plain epilogue.
template <typename Acc, bool ZeroRows = false>
__device__ __forceinline__ void finish_row(int64_t u, Acc sum, const Epi& e, const IterParams& p) {
    if (e.store_only) {  // dynamic repair: the level value only (and its FP32 rounding at a transition)
        if constexpr (sizeof(Acc) == 8) {
            const double sd = __dmul_rn(p.alpha, (double)sum);
            ((double*)e.y)[u] = sd;
            if (e.s32) e.s32[u] = f64_to_f32_rn(sd);
        } else {
            ((float*)e.y)[u] = __fmul_rn(p.alpha_f, (float)sum);
        }
        return;
    }
    double sd, c64, c32 = 0.0;
    bool zero = false;  // ZeroRows: a node without walks so far, every value of the row is +0
    if constexpr (sizeof(Acc) == 8) {
        const double c_prev = e.c64[u];
        if (ZeroRows && __double_as_longlong((double)sum) == 0 && __double_as_longlong(c_prev) == 0) {
            sd = 0.0;
            c64 = 0.0;
            zero = true;
            ((double*)e.y)[u] = 0.0;
            if (e.s32) e.s32[u] = 0.0f;
        } else {
            sd = __dmul_rn(p.alpha, (double)sum);
            ((double*)e.y)[u] = sd;
            if (e.s32) e.s32[u] = f64_to_f32_rn(sd);  // one rounding per row, not per gathered arc
            c64 = __dadd_rn(c_prev, sd);
            e.c64[u] = c64;
        }
        if (e.c32) c32 = e.c32[u];
    } else {
        const float sf = __fmul_rn(p.alpha_f, (float)sum);
        ((float*)e.y)[u] = sf;
        sd = f32_to_f64(sf);
        c32 = __dadd_rn(e.c32[u], sd);
        e.c32[u] = c32;
        c64 = e.c64[u];
    }
    if (e.active[u]) {
        double l = 0.0, up = 0.0;  // zero: c = s = +0, both bounds are +0 in either mode
        if (!ZeroRows || !zero || __double_as_longlong(c32) != 0) node_bounds(c64, c32, sd, p, e.bs, l, up);
        if (p.cert) {  // both the new and the stored bounds are valid: keep the tighter ones
            l = nn_max(l, e.lb[u]);
            up = nn_min(up, e.ub[u]);
        }
        e.lb[u] = l;  // read by the deactivation count of this level
        e.ub[u] = up;
        if (__double_as_longlong(l) >= __double_as_longlong(e.theta_prev)) {
            // one atomic per group of lanes that append together
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&e.ctrl->n_cand, (unsigned long long)grp.size());
            const unsigned long long pos = grp.shfl(base, 0) + grp.thread_rank();
            if (pos < (unsigned long long)e.cand_cap) {
                e.cand_l[pos] = l;
                e.cand_u[pos] = up;
                e.cand_id[pos] = e.perm[u];
            }
        }
    }
}

template <typename Acc>
__device__ __forceinline__ Acc addA(Acc a, Acc b);
template <>
__device__ __forceinline__ float addA<float>(float a, float b) { return __fadd_rn(a, b); }

// ---------------------------------------------------------------------------
// Exact accumulation of non-negative doubles.
//
// A term x = m * 2^(e - 1075) (m < 2^53 its integer mantissa, e >= 1 its
// biased exponent, e = 1 for subnormals and zero) is added to
// W * 2^(E - 1075 - XF), W a 128-bit integer in four 32-bit words and E the
// largest exponent the accumulator has seen, as the integer
// m * 2^(XF - (E - e)).  With XF = 31 a term with E - e <= 31 spans at most
// three words after its shift, so the common case is three funnel shifts and
// one carry chain; a term more than 2^31 below E is truncated at W's last
// bit (slow path), and a larger exponent shifts W right (slow path).  W stays
// below 2^85 per 2^1 terms of the top binade, so no sum of a row can carry
// out of 128 bits.  E = 0 marks an empty accumulator.
// ---------------------------------------------------------------------------
constexpr int XF = 31;

struct XAcc {
    uint32_t w0, w1, w2, w3;
    int E;
};

__device__ __forceinline__ XAcc xacc_zero() { return XAcc{0u, 0u, 0u, 0u, 0}; }

__device__ __forceinline__ unsigned long long lo64(const XAcc& a) {
    return ((unsigned long long)a.w1 << 32) | a.w0;
}
__device__ __forceinline__ unsigned long long hi64(const XAcc& a) {
    return ((unsigned long long)a.w3 << 32) | a.w2;
}
__device__ __forceinline__ void set128(XAcc& a, unsigned long long lo, unsigned long long hi) {
    a.w0 = (uint32_t)lo;
    a.w1 = (uint32_t)(lo >> 32);
    a.w2 = (uint32_t)hi;
    a.w3 = (uint32_t)(hi >> 32);
}

// W >>= d (truncating), d >= 0
__device__ __forceinline__ void shr128(XAcc& a, int d) {
    if (d <= 0) return;
    unsigned long long lo = lo64(a), hi = hi64(a);
    if (d >= 128) {
        lo = 0ull;
        hi = 0ull;
    } else if (d >= 64) {
        lo = hi >> (d - 64);
        hi = 0ull;
    } else {
        lo = (lo >> d) | (hi << (64 - d));
        hi >>= d;
    }
    set128(a, lo, hi);
}

// W += (p2:p1:p0)
__device__ __forceinline__ void add96(XAcc& a, uint32_t p0, uint32_t p1, uint32_t p2) {
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"(p0), "r"(p1), "r"(p2));
}

// W += V (128 bits)
__device__ __forceinline__ void add128(XAcc& a, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"(v0), "r"(v1), "r"(v2), "r"(v3));
}

__device__ __forceinline__ int exp_of(double x) { return max((int)((uint32_t)__double2hiint(x) >> 20), 1); }

// the rare cases of xacc_add: E < e (rescale first) or E - e > XF (truncate)
__device__ __noinline__ XAcc xacc_add_slow(XAcc a, int e, uint32_t m0, uint32_t m1) {
    int d = a.E - e;
    if (d < 0) {
        shr128(a, -d);
        a.E = e;
        d = 0;
    }
    if (d <= XF) {
        const uint32_t sh = (uint32_t)(XF - d);
        add96(a, m0 << sh, __funnelshift_l(m0, m1, sh), __funnelshift_l(m1, 0u, sh));
    } else {
        const int rs = d - XF;  // m * 2^-rs, truncated
        if (rs < 53) {
            const unsigned long long m = (((unsigned long long)m1 << 32) | m0) >> rs;
            add96(a, (uint32_t)m, (uint32_t)(m >> 32), 0u);
        }
    }
    return a;
}

// The fast path takes a normal term within XF binades below E; a zero term
// (padding) adds nothing; the rest (rescale, truncation, subnormals, whose
// exponent counts as 1 and whose mantissa has no implicit bit) goes through
// xacc_add_slow, which gives the fast path's result wherever both apply.
__device__ __forceinline__ void xacc_add(XAcc& a, double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t eb = hi >> 20;
    const uint32_t d = (uint32_t)(a.E - (int)eb);
    if (d <= (uint32_t)XF && eb != 0u) {
        const uint32_t m1 = (hi & 0xFFFFFu) | 0x100000u;
        const uint32_t sh = (uint32_t)XF - d;
        add96(a, lo << sh, __funnelshift_l(lo, m1, sh), __funnelshift_l(m1, 0u, sh));
    } else if ((hi | lo) != 0u) {
        a = xacc_add_slow(a, eb ? (int)eb : 1, lo, (hi & 0xFFFFFu) | (eb ? 0x100000u : 0u));
    }
}

// a += b (any exponents)
__device__ __forceinline__ void xacc_merge(XAcc& a, XAcc b) {
    if (b.E > a.E) {
        const XAcc t = a;
        a = b;
        b = t;
    }
    shr128(b, a.E - b.E);
    add128(a, b.w0, b.w1, b.w2, b.w3);
}

// Sum over groups of `width` lanes (8 or 32): every lane aligns to the
// group's largest exponent, then the aligned integers meet in a shuffle tree.
template <int width>
__device__ __forceinline__ XAcc xacc_group_sum(XAcc a) {
    int E = a.E;
    if constexpr (width == 32) {
        E = __reduce_max_sync(FULL, E);
    } else {
#pragma unroll
        for (int off = width / 2; off; off >>= 1) E = max(E, __shfl_xor_sync(FULL, E, off, width));
    }
    shr128(a, E - a.E);
    a.E = E;
#pragma unroll
    for (int off = width / 2; off; off >>= 1) {
        const uint32_t v0 = __shfl_down_sync(FULL, a.w0, off, width);
        const uint32_t v1 = __shfl_down_sync(FULL, a.w1, off, width);
        const uint32_t v2 = __shfl_down_sync(FULL, a.w2, off, width);
        const uint32_t v3 = __shfl_down_sync(FULL, a.w3, off, width);
        add128(a, v0, v1, v2, v3);
    }
    return a;
}

// W * 2^(E - 1075 - XF) rounded to the nearest double (ties to even)
__device__ __forceinline__ double xacc_to_double(const XAcc& a) {
    const unsigned long long L = lo64(a), H = hi64(a);
    if ((L | H) == 0ull) return 0.0;
    const int p = H ? 127 - __clzll((long long)H) : 63 - __clzll((long long)L);  // top bit
    int be = p - 52 + a.E - XF;
    unsigned long long T;
    bool rnd = false, sticky = false;
    if (p <= 52) {
        T = L << (52 - p);
    } else {
        const int sft = p - 52;  // 1..75
        const int rb = sft - 1;  // round bit; sticky = the bits below it
        if (rb < 64) {
            rnd = (L >> rb) & 1ull;
            sticky = rb ? (L & ((1ull << rb) - 1ull)) != 0ull : false;
        } else {
            rnd = (H >> (rb - 64)) & 1ull;
            sticky = L != 0ull || (rb > 64 && (H & ((1ull << (rb - 64)) - 1ull)) != 0ull);
        }
        XAcc t = a;
        shr128(t, sft);
        T = lo64(t);
    }
    if (rnd && (sticky || (T & 1ull))) {
        T += 1ull;
        if (T >> 53) {
            T >>= 1;
            be += 1;
        }
    }
    if (be >= 1) return __longlong_as_double((long long)(((unsigned long long)be << 52) | (T & 0xFFFFFFFFFFFFFull)));
    return ldexp((double)T, be - 1075);  // subnormal result
}

// Exact sum of x[col[j]] for j in [a, b) with stride `step` from a + first:
// groups of G loads in flight (past the end: zero, which the fast path adds
// as nothing).  G = 8 for rows whose lanes see many terms, G = 4 for short
// rows (fewer padded slots).  An empty accumulator starts at the largest
// exponent of its first group, so it rarely has to rescale.
// S: entries of x are S apart (S = 2: one state of the interleaved pairs of
// the two-state pass below).
template <int G, int S = 1>
__device__ __forceinline__ XAcc strided_xsum(const int32_t* __restrict__ col, const double* __restrict__ x,
                                             int64_t a, int64_t b, int first, int step) {
    XAcc s = xacc_zero();
    for (int64_t j = a + first; j < b; j += G * (int64_t)step) {
        double v[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int64_t jj = j + (int64_t)q * step;
            v[q] = jj < b ? __ldg(x + (int64_t)S * col[jj]) : 0.0;
        }
        if (s.E == 0) {
            int em = exp_of(v[0]);
#pragma unroll
            for (int q = 1; q < G; ++q) em = max(em, exp_of(v[q]));
            s.E = em;
        }
#pragma unroll
        for (int q = 0; q < G; ++q) xacc_add(s, v[q]);
    }
    return s;
}

// chunk partials: three words per chunk (W low, W high, E) for FP64 levels;
// the first word holds the FP32 sum (exact in FP64) for FP32 levels
__device__ __forceinline__ void store_part(double* part, int64_t ch, const XAcc& a) {
    unsigned long long* w = (unsigned long long*)part + 3 * ch;
    w[0] = lo64(a);
    w[1] = hi64(a);
    w[2] = (unsigned long long)(unsigned)a.E;
}

__device__ __forceinline__ XAcc load_part(const double* part, int64_t ch) {
    const unsigned long long* w = (const unsigned long long*)part + 3 * ch;
    XAcc a;
    set128(a, w[0], w[1]);
    a.E = (int)w[2];
    return a;
}

// The partials of chunks [first, first + count) merged by one warp: lane l
// merges chunks first + l, first + l + 32, ... in order, then the lanes meet.
// A chunk partial stays below 2^95 (2048 terms below 2^84), a lane's merge
// below 2^108 for any row that fits in memory, so 32 lanes cannot carry out.
__device__ __forceinline__ XAcc merge_chunks_warp(const double* __restrict__ part, int64_t first, int64_t count) {
    XAcc t = xacc_zero();
    for (int64_t q = threadIdx.x & 31; q < count; q += 32) xacc_merge(t, load_part(part, first + q));
    return xacc_group_sum<32>(t);
}

// Sum of x[col[j]] for j in [a, b) with stride `step` from a + first: eight
// loads in flight, each group of eight added as a pairwise tree (depth 3),
// groups chained in index order.
template <typename Tin, typename Acc, int S = 1>
__device__ __forceinline__ Acc strided_sum(const int32_t* __restrict__ col, const Tin* __restrict__ x, int64_t a,
                                           int64_t b, int first, int step) {
    Acc s = (Acc)0;
    for (int64_t j = a + first; j < b; j += 8 * (int64_t)step) {
        Acc v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t jj = j + (int64_t)q * step;
            v[q] = jj < b ? (Acc)__ldg(x + (int64_t)S * col[jj]) : (Acc)0;
        }
        const Acc t = addA<Acc>(addA<Acc>(addA<Acc>(v[0], v[1]), addA<Acc>(v[2], v[3])),
                                addA<Acc>(addA<Acc>(v[4], v[5]), addA<Acc>(v[6], v[7])));
        s = addA<Acc>(s, t);
    }
    return s;
}

// One level: Tin = type of level r-1, Tout = type of level r.  FP64 levels
// sum exactly (XAcc); FP32 levels add in FP32 (fixed pairwise order).
template <typename Off, typename Tin, typename Tout>
__device__ __forceinline__ void spmv_rows(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                          const SpmvLayout& L, const Tin* __restrict__ x, const Epi& ep,
                                          const int32_t* __restrict__ chunk_row,
                                          const int64_t* __restrict__ chunk_first, double* chunk_part,
                                          const IterParams& p) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t b = blockIdx.x;
    if constexpr (sizeof(Tout) == 8) {
        static_assert(sizeof(Tin) == 8, "FP64 levels follow FP64 levels");
        if (b >= L.blk_thread) {  // THREAD rows
            const int64_t u = L.row_thread + (b - L.blk_thread) * BLOCK + tid;
            if (u < L.n) finish_row<double>(u, xacc_to_double(strided_xsum<4>(col, x, rowptr[u], rowptr[u + 1], 0, 1)), ep, p);
        } else if (b >= L.blk_octet) {  // OCTET rows
            const int64_t u = L.row_octet + (b - L.blk_octet) * (BLOCK / 8) + (tid >> 3);
            const int sub = tid & 7;
            XAcc s = xacc_zero();
            if (u < L.row_thread) s = strided_xsum<4>(col, x, rowptr[u], rowptr[u + 1], sub, 8);
            s = xacc_group_sum<8>(s);
            if (sub == 0 && u < L.row_thread) finish_row<double>(u, xacc_to_double(s), ep, p);
        } else if (b >= L.blk_warp) {  // WARP rows
            const int64_t u = L.row_warp + (b - L.blk_warp) * WARPS + wid;
            XAcc s = xacc_zero();
            if (u < L.row_octet) s = strided_xsum<8>(col, x, rowptr[u], rowptr[u + 1], lane, 32);
            s = xacc_group_sum<32>(s);
            if (lane == 0 && u < L.row_octet) finish_row<double>(u, xacc_to_double(s), ep, p);
        } else {  // CHUNK rows: one warp per chunk of CHUNK_ARCS arcs
            const int64_t ch = b * WARPS + wid;
            XAcc s = xacc_zero();
            if (ch < L.chunks) {
                const int64_t u = chunk_row[ch];
                const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
                const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
                s = strided_xsum<8>(col, x, j0, j1, lane, 32);
            }
            s = xacc_group_sum<32>(s);
            if (lane == 0 && ch < L.chunks) store_part(chunk_part, ch, s);
        }
    } else {
        typedef float Acc;
        if (b >= L.blk_thread) {  // THREAD rows
            const int64_t u = L.row_thread + (b - L.blk_thread) * BLOCK + tid;
            if (u < L.n) finish_row<Acc>(u, strided_sum<Tin, Acc>(col, x, rowptr[u], rowptr[u + 1], 0, 1), ep, p);
        } else if (b >= L.blk_octet) {  // OCTET rows
            const int64_t u = L.row_octet + (b - L.blk_octet) * (BLOCK / 8) + (tid >> 3);
            const int sub = tid & 7;
            Acc s = (Acc)0;
            if (u < L.row_thread) s = strided_sum<Tin, Acc>(col, x, rowptr[u], rowptr[u + 1], sub, 8);
#pragma unroll
            for (int off = 4; off; off >>= 1) s = addA<Acc>(s, __shfl_down_sync(FULL, s, off, 8));
            if (sub == 0 && u < L.row_thread) finish_row<Acc>(u, s, ep, p);
        } else if (b >= L.blk_warp) {  // WARP rows
            const int64_t u = L.row_warp + (b - L.blk_warp) * WARPS + wid;
            Acc s = (Acc)0;
            if (u < L.row_octet) s = strided_sum<Tin, Acc>(col, x, rowptr[u], rowptr[u + 1], lane, 32);
#pragma unroll
            for (int off = 16; off; off >>= 1) s = addA<Acc>(s, __shfl_down_sync(FULL, s, off));
            if (lane == 0 && u < L.row_octet) finish_row<Acc>(u, s, ep, p);
        } else {  // CHUNK rows: one warp per chunk of CHUNK_ARCS arcs
            const int64_t ch = b * WARPS + wid;
            Acc s = (Acc)0;
            if (ch < L.chunks) {
                const int64_t u = chunk_row[ch];
                const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
                const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
                s = strided_sum<Tin, Acc>(col, x, j0, j1, lane, 32);
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) s = addA<Acc>(s, __shfl_down_sync(FULL, s, off));
            if (lane == 0 && ch < L.chunks) chunk_part[3 * ch] = (double)s;  // exact for FP32 sums
        }
    }
}

// FP32-certified mode: s32 holds the last FP64 level rounded to FP32, the
// input of the first FP32 level.  A ranking writes it at every FP64 level
// while the switch is ahead; a repair (store_level > 0) rewrites it at that
// last FP64 level, min(f32_from - 1, r) for the r levels held.
__device__ __forceinline__ bool writes_s32(const Ctrl* ctrl, const IterParams& p, int r_cur, int store_level) {
    if (!p.cert) return false;
    if (!store_level) return r_cur < ctrl->f32_from;
    return r_cur == min(ctrl->f32_from - 1, ctrl->r);
}

__device__ __forceinline__ Epi make_epi(void* y, double* c64, double* c32, double* lb, double* ub, uint8_t* active,
                                        const int32_t* perm, double* cand_l, double* cand_u, int32_t* cand_id,
                                        int64_t cand_cap, Ctrl* ctrl, const IterParams& p, float* s32 = nullptr) {
    return Epi{y,    c64,     c32,      lb,   ub, active, perm, cand_l, cand_u, cand_id, cand_cap, ctrl,
               ctrl->theta_prev, bstate(ctrl, p), 0, s32};
}

// Level 1 of a ranking as one pass over all rows, any row mode: s_0 = 1, so
// the exact sum of a row is its length (A 1 = deg) and no walk value is read;
// s_1 = alpha deg goes through the epilogue of every level, in a grid sized
// for O(n) work (no chunk partials: no fixup follows).  The bits are those a
// gather level would give: an exact sum of ones, rounded once.
template <typename Off>
__global__ void degree_level_kernel(const Off* __restrict__ rowptr, int64_t n, double* walk, double* c64,
                                    double* c32, double* lb, double* ub, uint8_t* active,
                                    const int32_t* __restrict__ perm, double* cand_l, double* cand_u,
                                    int32_t* cand_id, int64_t cand_cap, float* s32, Ctrl* ctrl, IterParams p) {
    if (ctrl->stop) return;
    const Epi ep = make_epi(walk_slot(walk, p, 1), c64, c32, lb, ub, active, perm, cand_l, cand_u, cand_id,
                            cand_cap, ctrl, p, (p.cert && 1 < ctrl->f32_from) ? s32 : nullptr);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        finish_row<double, true>(u, (double)((int64_t)rowptr[u + 1] - (int64_t)rowptr[u]), ep, p);
}

// Six 256-thread blocks per SM (40 registers): the gathers need the warps in
// flight more than the lanes need registers.
template <typename Off>
__global__ void __launch_bounds__(BLOCK, 6)
spmv_rows_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, SpmvLayout L, double* walk,
                 double* c64, double* c32, double* lb, double* ub, uint8_t* active, const int32_t* __restrict__ perm,
                 const int32_t* __restrict__ chunk_row, const int64_t* __restrict__ chunk_first, double* chunk_part,
                 double* cand_l, double* cand_u, int32_t* cand_id, int64_t cand_cap, float* s32, Ctrl* ctrl,
                 IterParams p, int store_level) {
    // store_level > 0: dynamic repair of one level, s only
    if (!store_level && ctrl->stop) return;
    const int r_cur = store_level ? store_level : ctrl->r + 1;
    const int f32_from = ctrl->f32_from;
    const double* xs = walk_slot(walk, p, r_cur - 1);
    double* ys = walk_slot(walk, p, r_cur);
    Epi ep = make_epi(ys, c64, c32, lb, ub, active, perm, cand_l, cand_u, cand_id, cand_cap, ctrl, p,
                      writes_s32(ctrl, p, r_cur, store_level) ? s32 : nullptr);
    ep.store_only = store_level > 0;
    if (r_cur < f32_from)  // level 1, when it comes here, gathers s_0 = 1 (f32_from >= 2)
        spmv_rows<Off, double, double>(rowptr, col, L, xs, ep, chunk_row, chunk_first, chunk_part, p);
    else if (r_cur == f32_from)
        spmv_rows<Off, float, float>(rowptr, col, L, s32, ep, chunk_row, chunk_first, chunk_part, p);
    else
        spmv_rows<Off, float, float>(rowptr, col, L, (const float*)xs, ep, chunk_row, chunk_first, chunk_part, p);
}

// CHUNK rows of an FP32 level: the chunk sums of a row, in groups of 64, each
// group a pairwise tree in FP32 (level by level, entry q = entry 2q + entry
// 2q+1), the group totals chained in order.  A warp per row: lane l holds
// entry l of each tree level, partners come by shuffle.
__device__ __forceinline__ float chunk_tree_warp(const double* __restrict__ part, int64_t first, int64_t count) {
    const int lane = threadIdx.x & 31;
    float total = 0.0f;
    for (int64_t base = 0; base < count; base += 64) {
        const int64_t m = min((int64_t)64, count - base);
        const int q0 = 2 * lane, q1 = 2 * lane + 1;
        const float a = q0 < m ? (float)part[3 * (first + base + q0)] : 0.0f;  // FP32 sums, exact in FP64
        const float b = q1 < m ? (float)part[3 * (first + base + q1)] : 0.0f;
        float v = __fadd_rn(a, b);
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {  // entries q >= w of a level are not used further
            const float x = __shfl_sync(FULL, v, (2 * lane) & 31);
            const float y = __shfl_sync(FULL, v, (2 * lane + 1) & 31);
            v = __fadd_rn(x, y);
        }
        total = __fadd_rn(total, __shfl_sync(FULL, v, 0));
    }
    return total;
}

// CHUNK rows: one warp per row merges the row's chunk partials, then its
// first lane finishes the row.
__global__ void spmv_chunk_fixup(SpmvLayout L, double* walk, double* c64, double* c32, double* lb, double* ub,
                                 uint8_t* active,
                                 const int32_t* __restrict__ perm, const int64_t* __restrict__ chunk_first,
                                 const double* __restrict__ chunk_part, double* cand_l, double* cand_u,
                                 int32_t* cand_id, int64_t cand_cap, float* s32, Ctrl* ctrl, IterParams p,
                                 int store_level) {
    if (!store_level && ctrl->stop) return;
    const int r_cur = store_level ? store_level : ctrl->r + 1;
    double* ys = walk_slot(walk, p, r_cur);
    Epi ep = make_epi(ys, c64, c32, lb, ub, active, perm, cand_l, cand_u, cand_id, cand_cap, ctrl, p,
                      writes_s32(ctrl, p, r_cur, store_level) ? s32 : nullptr);
    ep.store_only = store_level > 0;
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;  // one warp per CHUNK row
    if (u >= L.row_warp) return;
    const int64_t first = chunk_first[u], count = chunk_first[u + 1] - first;
    if (r_cur < ctrl->f32_from) {
        const XAcc t = merge_chunks_warp(chunk_part, first, count);
        if ((threadIdx.x & 31) == 0) finish_row<double>(u, xacc_to_double(t), ep, p);
    } else {
        const float t = chunk_tree_warp(chunk_part, first, count);
        if ((threadIdx.x & 31) == 0) finish_row<float>(u, t, ep, p);
    }
}

}  // namespace

// Longest chain of additions in one row sum: ceil(per-lane terms / 8) chained
// groups + 3 (tree of 8) + shuffle levels + tree over chunks.  The row modes
// are fixed by position; their nominal degree limits (16, 128, 2048) hold at
// creation, and an update batch can push a row past its mode's limit
// (sum_depth_of with the largest degrees seen in each mode).
int sum_depth_of(int64_t deg_thread, int64_t deg_octet, int64_t deg_warp, bool has_octet, bool has_warp,
                 int64_t max_chunks_per_row) {
    auto lane_depth = [](int64_t terms) { return (int)std::min<int64_t>((terms + 7) / 8 + 3, 1 << 24); };
    int d = lane_depth(std::max<int64_t>(deg_thread, 16));                               // THREAD
    if (has_octet) d = std::max(d, lane_depth((std::max<int64_t>(deg_octet, 128) + 7) / 8) + 3);   // OCTET
    if (has_warp) d = std::max(d, lane_depth((std::max<int64_t>(deg_warp, 2048) + 31) / 32) + 5);  // WARP
    if (max_chunks_per_row > 0)  // CHUNK: + tree of 64 + chained groups
        d = std::max(d, lane_depth(CHUNK_ARCS / 32) + 5 + 6 + (int)((max_chunks_per_row + 63) / 64));
    return d;
}

int max_sum_depth(const SpmvLayout& L, int64_t max_chunks_per_row) {
    return sum_depth_of(16, 128, 2048, L.row_thread > L.row_octet, L.row_octet > L.row_warp,
                        L.row_warp > 0 ? std::max<int64_t>(max_chunks_per_row, 1) : 0);
}

static cudaError_t spmv_launch(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int store_level,
                               cudaStream_t st) {
    const SpmvLayout& L = g.layout;
    if (L.blocks_total > 0) {
        if (g.off64)
            spmv_rows_kernel<int64_t><<<(unsigned)L.blocks_total, BLOCK, 0, st>>>(
                (const int64_t*)g.rowptr, g.col, L, (double*)b.walk, b.c, b.c32, b.lb, b.ub, b.active, g.perm,
                g.chunk_row, g.chunk_first, g.chunk_part, b.cand_l, b.cand_u, b.cand_id, b.cand_cap, b.s32, b.ctrl, p,
                store_level);
        else
            spmv_rows_kernel<int32_t><<<(unsigned)L.blocks_total, BLOCK, 0, st>>>(
                (const int32_t*)g.rowptr, g.col, L, (double*)b.walk, b.c, b.c32, b.lb, b.ub, b.active, g.perm,
                g.chunk_row, g.chunk_first, g.chunk_part, b.cand_l, b.cand_u, b.cand_id, b.cand_cap, b.s32, b.ctrl, p,
                store_level);
    }
    if (L.row_warp > 0)
        spmv_chunk_fixup<<<(unsigned)((L.row_warp * 32 + 127) / 128), 128, 0, st>>>(
            L, (double*)b.walk, b.c, b.c32, b.lb, b.ub, b.active, g.perm, g.chunk_first, g.chunk_part, b.cand_l,
            b.cand_u, b.cand_id, b.cand_cap, b.s32, b.ctrl, p, store_level);
    return cudaGetLastError();
}

cudaError_t launch_spmv(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, bool fp32,
                        cudaStream_t st) {
    (void)fp32;
    return spmv_launch(g, b, p, 0, st);
}

namespace {
__global__ void convert_kernel(const double* __restrict__ in, int64_t n, float* out, double* back) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float f = f64_to_f32_rn(in[i]);
        out[i] = f;
        back[i] = f32_to_f64(f);
    }
}
}  // namespace

cudaError_t launch_convert(const double* in, int64_t n, float* out, double* back, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
    convert_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, n, out, back);
    return cudaGetLastError();
}

namespace {
template <typename Off>
__global__ void degree_store_kernel(const Off* __restrict__ rowptr, int64_t n, double* walk, float* s32,
                                    const Ctrl* ctrl, IterParams p) {
    double* y = walk_slot(walk, p, 1);
    float* t = writes_s32(ctrl, p, 1, 1) ? s32 : nullptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const double sd = __dmul_rn(p.alpha, (double)((int64_t)rowptr[u + 1] - (int64_t)rowptr[u]));
        y[u] = sd;
        if (t) t[u] = f64_to_f32_rn(sd);
    }
}
}  // namespace

cudaError_t launch_degree_store(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>(std::max<int64_t>((g.n + BLOCK - 1) / BLOCK, 1), 152 * 8);
    if (g.off64)
        degree_store_kernel<int64_t><<<(unsigned)blocks, BLOCK, 0, st>>>((const int64_t*)g.rowptr, g.n,
                                                                         (double*)b.walk, b.s32, b.ctrl, p);
    else
        degree_store_kernel<int32_t><<<(unsigned)blocks, BLOCK, 0, st>>>((const int32_t*)g.rowptr, g.n,
                                                                         (double*)b.walk, b.s32, b.ctrl, p);
    return cudaGetLastError();
}

cudaError_t launch_degree_level(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>(std::max<int64_t>((g.n + BLOCK - 1) / BLOCK, 1), 152 * 8);
    if (g.off64)
        degree_level_kernel<int64_t><<<(unsigned)blocks, BLOCK, 0, st>>>(
            (const int64_t*)g.rowptr, g.n, (double*)b.walk, b.c, b.c32, b.lb, b.ub, b.active, g.perm, b.cand_l,
            b.cand_u, b.cand_id, b.cand_cap, b.s32, b.ctrl, p);
    else
        degree_level_kernel<int32_t><<<(unsigned)blocks, BLOCK, 0, st>>>(
            (const int32_t*)g.rowptr, g.n, (double*)b.walk, b.c, b.c32, b.lb, b.ub, b.active, g.perm, b.cand_l,
            b.cand_u, b.cand_id, b.cand_cap, b.s32, b.ctrl, p);
    return cudaGetLastError();
}

cudaError_t launch_spmv_store(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int level,
                              cudaStream_t st) {
    return spmv_launch(g, b, p, level, st);
}

// One warp per listed row: the row's s_level recomputed with the lane
// partition spmv_rows_kernel uses for that row (its row mode is set by its
// internal index) and the same merges, so a repaired level has the bits of a
// full recomputation.  CHUNK rows are left to the two hub kernels below,
// which split them over warps as the SpMV does.
template <typename Off>
__global__ void rows_store_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, SpmvLayout L,
                                  const int32_t* __restrict__ rows, const unsigned long long* nrows_ptr,
                                  double* walk, float* s32, const Ctrl* ctrl, IterParams p, int level) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t nrows = (int64_t)*nrows_ptr;
    const int f32_from = ctrl->f32_from;
    if (level >= f32_from) {  // FP32 level: the FP32 order of spmv_rows
        const float* __restrict__ x = level == f32_from ? s32 : (const float*)walk_slot(walk, p, level - 1);
        float* y = (float*)walk_slot(walk, p, level);
        for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < nrows; w += warps) {
            const int64_t u = rows[w];
            if (u < L.row_warp) continue;  // CHUNK row
            const int64_t a = rowptr[u], e = rowptr[u + 1];
            float s = 0.0f;
            if (u >= L.row_thread) {
                if (lane == 0) s = strided_sum<float, float>(col, x, a, e, 0, 1);
            } else if (u >= L.row_octet) {
                if (lane < 8) s = strided_sum<float, float>(col, x, a, e, lane, 8);
#pragma unroll
                for (int off = 4; off; off >>= 1) s = addA<float>(s, __shfl_down_sync(FULL, s, off, 8));
            } else {
                s = strided_sum<float, float>(col, x, a, e, lane, 32);
#pragma unroll
                for (int off = 16; off; off >>= 1) s = addA<float>(s, __shfl_down_sync(FULL, s, off));
            }
            if (lane == 0) y[u] = __fmul_rn(p.alpha_f, s);
        }
        return;
    }
    const double* __restrict__ x = walk_slot(walk, p, level - 1);
    double* y = walk_slot(walk, p, level);
    float* t = writes_s32(ctrl, p, level, level) ? s32 : nullptr;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < nrows; w += warps) {
        const int64_t u = rows[w];
        if (u < L.row_warp) continue;     // CHUNK row
        const int64_t a = rowptr[u], e = rowptr[u + 1];
        XAcc s = xacc_zero();
        if (u >= L.row_thread) {          // THREAD: lane 0 alone, step 1
            if (lane == 0) s = strided_xsum<4>(col, x, a, e, 0, 1);
        } else if (u >= L.row_octet) {    // OCTET: lanes 0..7, step 8
            if (lane < 8) s = strided_xsum<4>(col, x, a, e, lane, 8);
            s = xacc_group_sum<8>(s);
        } else {                          // WARP
            s = strided_xsum<8>(col, x, a, e, lane, 32);
            s = xacc_group_sum<32>(s);
        }
        if (lane == 0) {
            const double sd = __dmul_rn(p.alpha, xacc_to_double(s));
            y[u] = sd;
            if (t) t[u] = f64_to_f32_rn(sd);
        }
    }
}

__device__ __forceinline__ bool visited(const uint32_t* vbits, int64_t u) {
    return (vbits[u >> 5] >> (u & 31)) & 1u;
}

// chunk partials of the CHUNK rows in the frontier (one warp per chunk)
template <typename Off>
__global__ void hub_chunks_store_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, SpmvLayout L,
                                        const int32_t* __restrict__ chunk_row,
                                        const int64_t* __restrict__ chunk_first, double* chunk_part,
                                        const uint32_t* __restrict__ vbits, const double* walk,
                                        const float* __restrict__ s32, const Ctrl* ctrl, IterParams p, int level) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int f32_from = ctrl->f32_from;
    const double* __restrict__ x = walk_slot(walk, p, level - 1);
    const float* __restrict__ xf = level == f32_from ? s32 : (const float*)x;
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < L.chunks; ch += warps) {
        const int64_t u = chunk_row[ch];
        if (!visited(vbits, u)) continue;
        const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
        const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
        if (level >= f32_from) {  // FP32 level: the chunk sum of spmv_rows, exact in FP64
            float s = strided_sum<float, float>(col, xf, j0, j1, lane, 32);
#pragma unroll
            for (int off = 16; off; off >>= 1) s = addA<float>(s, __shfl_down_sync(FULL, s, off));
            if (lane == 0) chunk_part[3 * ch] = (double)s;
        } else {
            const XAcc t = xacc_group_sum<32>(strided_xsum<8>(col, x, j0, j1, lane, 32));
            if (lane == 0) store_part(chunk_part, ch, t);
        }
    }
}

// the CHUNK rows in the frontier: partials merged as spmv_chunk_fixup merges them
__global__ void hub_rows_store_kernel(SpmvLayout L, const int64_t* __restrict__ chunk_first,
                                      const double* __restrict__ chunk_part, const uint32_t* __restrict__ vbits,
                                      double* walk, float* s32, const Ctrl* ctrl, IterParams p, int level) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;  // one warp per CHUNK row
    if (u >= L.row_warp || !visited(vbits, u)) return;
    const int64_t first = chunk_first[u], count = chunk_first[u + 1] - first;
    if (level >= ctrl->f32_from) {  // FP32 level: the chunk tree of spmv_chunk_fixup
        const float t = chunk_tree_warp(chunk_part, first, count);
        if ((threadIdx.x & 31) == 0) ((float*)walk_slot(walk, p, level))[u] = __fmul_rn(p.alpha_f, t);
        return;
    }
    const XAcc t = merge_chunks_warp(chunk_part, first, count);
    if ((threadIdx.x & 31) == 0) {
        const double sd = __dmul_rn(p.alpha, xacc_to_double(t));
        walk_slot(walk, p, level)[u] = sd;
        if (writes_s32(ctrl, p, level, level)) s32[u] = f64_to_f32_rn(sd);
    }
}

cudaError_t launch_rows_store(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, const int32_t* rows,
                              const unsigned long long* nrows_dev, int64_t nrows_max, const uint32_t* vbits,
                              int level, cudaStream_t st) {
    if (nrows_max <= 0) return cudaSuccess;
    int64_t blocks = (nrows_max + 7) / 8;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (g.off64)
        rows_store_kernel<int64_t><<<(unsigned)blocks, 256, 0, st>>>((const int64_t*)g.rowptr, g.col, g.layout, rows,
                                                                    nrows_dev, (double*)b.walk, b.s32, b.ctrl, p,
                                                                    level);
    else
        rows_store_kernel<int32_t><<<(unsigned)blocks, 256, 0, st>>>((const int32_t*)g.rowptr, g.col, g.layout, rows,
                                                                    nrows_dev, (double*)b.walk, b.s32, b.ctrl, p,
                                                                    level);
    const SpmvLayout& L = g.layout;
    if (L.chunks > 0) {
        const unsigned cb = (unsigned)std::min<int64_t>((L.chunks + 7) / 8, 152 * 32);
        if (g.off64)
            hub_chunks_store_kernel<int64_t><<<cb, 256, 0, st>>>((const int64_t*)g.rowptr, g.col, L, g.chunk_row,
                                                                g.chunk_first, g.chunk_part, vbits,
                                                                (const double*)b.walk, b.s32, b.ctrl, p, level);
        else
            hub_chunks_store_kernel<int32_t><<<cb, 256, 0, st>>>((const int32_t*)g.rowptr, g.col, L, g.chunk_row,
                                                                g.chunk_first, g.chunk_part, vbits,
                                                                (const double*)b.walk, b.s32, b.ctrl, p, level);
        hub_rows_store_kernel<<<(unsigned)((L.row_warp * 32 + 127) / 128), 128, 0, st>>>(
            L, g.chunk_first, g.chunk_part, vbits, (double*)b.walk, b.s32, b.ctrl, p, level);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Two graph states in one pass.
//
// A server with two batches of one graph queued answers both: A is the graph
// after the first batch, B the graph after the second.  On graphs whose
// repairs are whole levels (a batch reaches a hub within a level or two),
// the walk levels of A and B are computed together, over B's adjacency, with
// the level vectors of the two states stored interleaved: entry 2v is A's
// s_i(v), entry 2v + 1 is B's (16 bytes per node for FP64 levels, 8 for FP32
// ones).  One gathered line then serves both states, and the gathers, not
// the arithmetic, bound the level.  The rows the second batch changed have
// A's adjacency in A's graph: their A entries are recomputed afterwards from
// A's rows (pair_fix_*).  Each state's row sums use the lane partition, the
// grouping and the order of the one-state kernel, so every entry has the bits
// that a repair of that state alone gives.
// ---------------------------------------------------------------------------
namespace {

template <int G>
__device__ __forceinline__ void strided_xsum2(const int32_t* __restrict__ col, const double2* __restrict__ x,
                                              int64_t a, int64_t b, int first, int step, XAcc& sa, XAcc& sb) {
    sa = xacc_zero();
    sb = xacc_zero();
    for (int64_t j = a + first; j < b; j += G * (int64_t)step) {
        double2 v[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int64_t jj = j + (int64_t)q * step;
            v[q] = jj < b ? __ldg(x + col[jj]) : make_double2(0.0, 0.0);
        }
        if (sa.E == 0) {
            int em = exp_of(v[0].x);
#pragma unroll
            for (int q = 1; q < G; ++q) em = max(em, exp_of(v[q].x));
            sa.E = em;
        }
        if (sb.E == 0) {
            int em = exp_of(v[0].y);
#pragma unroll
            for (int q = 1; q < G; ++q) em = max(em, exp_of(v[q].y));
            sb.E = em;
        }
#pragma unroll
        for (int q = 0; q < G; ++q) xacc_add(sa, v[q].x);
#pragma unroll
        for (int q = 0; q < G; ++q) xacc_add(sb, v[q].y);
    }
}

__device__ __forceinline__ void strided_sum2(const int32_t* __restrict__ col, const float2* __restrict__ x, int64_t a,
                                             int64_t b, int first, int step, float& sa, float& sb) {
    sa = 0.0f;
    sb = 0.0f;
    for (int64_t j = a + first; j < b; j += 8 * (int64_t)step) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t jj = j + (int64_t)q * step;
            v[q] = jj < b ? __ldg(x + col[jj]) : make_float2(0.0f, 0.0f);
        }
        const float ta = __fadd_rn(__fadd_rn(__fadd_rn(v[0].x, v[1].x), __fadd_rn(v[2].x, v[3].x)),
                                   __fadd_rn(__fadd_rn(v[4].x, v[5].x), __fadd_rn(v[6].x, v[7].x)));
        const float tb = __fadd_rn(__fadd_rn(__fadd_rn(v[0].y, v[1].y), __fadd_rn(v[2].y, v[3].y)),
                                   __fadd_rn(__fadd_rn(v[4].y, v[5].y), __fadd_rn(v[6].y, v[7].y)));
        sa = __fadd_rn(sa, ta);
        sb = __fadd_rn(sb, tb);
    }
}

template <int width>
__device__ __forceinline__ float fsum_group(float s) {
#pragma unroll
    for (int off = width / 2; off; off >>= 1) s = __fadd_rn(s, __shfl_down_sync(FULL, s, off, width));
    return s;
}

// s_i of both states from their exact row sums; at the level whose FP32
// rounding feeds the first FP32 level, that rounding too
__device__ __forceinline__ void store_pair64(double2* y, float2* t, int64_t u, const XAcc& sa, const XAcc& sb,
                                             double alpha) {
    const double a = __dmul_rn(alpha, xacc_to_double(sa)), b = __dmul_rn(alpha, xacc_to_double(sb));
    y[u] = make_double2(a, b);
    if (t) t[u] = make_float2(f64_to_f32_rn(a), f64_to_f32_rn(b));
}

// Level `level` >= 2 of both states over B's adjacency (store only).  Levels
// below f32_from are FP64 (x and y double2), the others FP32 (float2; level
// f32_from reads the FP32 roundings t_in of the level before).  Four 256-thread
// blocks per SM: two accumulators per lane take the registers of the wider
// gathers.
template <typename Off>
__global__ void __launch_bounds__(BLOCK, 4)
spmv_pair_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, SpmvLayout L,
                 const int32_t* __restrict__ chunk_row, const int64_t* __restrict__ chunk_first, double* P,
                 int64_t pstride, int level, int f32_from, const float2* __restrict__ t_in, float2* t_out,
                 double* part_a, double* part_b, double alpha, float alpha_f) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t b = blockIdx.x;
    if (level < f32_from) {
        const double2* __restrict__ x = (const double2*)(P + (size_t)(level - 1) * pstride);
        double2* y = (double2*)(P + (size_t)level * pstride);
        XAcc sa, sb;
        if (b >= L.blk_thread) {
            const int64_t u = L.row_thread + (b - L.blk_thread) * BLOCK + tid;
            if (u < L.n) {
                strided_xsum2<4>(col, x, rowptr[u], rowptr[u + 1], 0, 1, sa, sb);
                store_pair64(y, t_out, u, sa, sb, alpha);
            }
        } else if (b >= L.blk_octet) {
            const int64_t u = L.row_octet + (b - L.blk_octet) * (BLOCK / 8) + (tid >> 3);
            const int sub = tid & 7;
            sa = xacc_zero();
            sb = xacc_zero();
            if (u < L.row_thread) strided_xsum2<4>(col, x, rowptr[u], rowptr[u + 1], sub, 8, sa, sb);
            sa = xacc_group_sum<8>(sa);
            sb = xacc_group_sum<8>(sb);
            if (sub == 0 && u < L.row_thread) store_pair64(y, t_out, u, sa, sb, alpha);
        } else if (b >= L.blk_warp) {
            const int64_t u = L.row_warp + (b - L.blk_warp) * WARPS + wid;
            sa = xacc_zero();
            sb = xacc_zero();
            if (u < L.row_octet) strided_xsum2<8>(col, x, rowptr[u], rowptr[u + 1], lane, 32, sa, sb);
            sa = xacc_group_sum<32>(sa);
            sb = xacc_group_sum<32>(sb);
            if (lane == 0 && u < L.row_octet) store_pair64(y, t_out, u, sa, sb, alpha);
        } else {
            const int64_t ch = b * WARPS + wid;
            sa = xacc_zero();
            sb = xacc_zero();
            if (ch < L.chunks) {
                const int64_t u = chunk_row[ch];
                const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
                const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
                strided_xsum2<8>(col, x, j0, j1, lane, 32, sa, sb);
            }
            sa = xacc_group_sum<32>(sa);
            sb = xacc_group_sum<32>(sb);
            if (lane == 0 && ch < L.chunks) {
                store_part(part_a, ch, sa);
                store_part(part_b, ch, sb);
            }
        }
    } else {
        const float2* __restrict__ x = level == f32_from ? t_in : (const float2*)(P + (size_t)(level - 1) * pstride);
        float2* y = (float2*)(P + (size_t)level * pstride);
        float sa = 0.0f, sb = 0.0f;
        if (b >= L.blk_thread) {
            const int64_t u = L.row_thread + (b - L.blk_thread) * BLOCK + tid;
            if (u < L.n) {
                strided_sum2(col, x, rowptr[u], rowptr[u + 1], 0, 1, sa, sb);
                y[u] = make_float2(__fmul_rn(alpha_f, sa), __fmul_rn(alpha_f, sb));
            }
        } else if (b >= L.blk_octet) {
            const int64_t u = L.row_octet + (b - L.blk_octet) * (BLOCK / 8) + (tid >> 3);
            const int sub = tid & 7;
            if (u < L.row_thread) strided_sum2(col, x, rowptr[u], rowptr[u + 1], sub, 8, sa, sb);
            sa = fsum_group<8>(sa);
            sb = fsum_group<8>(sb);
            if (sub == 0 && u < L.row_thread) y[u] = make_float2(__fmul_rn(alpha_f, sa), __fmul_rn(alpha_f, sb));
        } else if (b >= L.blk_warp) {
            const int64_t u = L.row_warp + (b - L.blk_warp) * WARPS + wid;
            if (u < L.row_octet) strided_sum2(col, x, rowptr[u], rowptr[u + 1], lane, 32, sa, sb);
            sa = fsum_group<32>(sa);
            sb = fsum_group<32>(sb);
            if (lane == 0 && u < L.row_octet) y[u] = make_float2(__fmul_rn(alpha_f, sa), __fmul_rn(alpha_f, sb));
        } else {
            const int64_t ch = b * WARPS + wid;
            if (ch < L.chunks) {
                const int64_t u = chunk_row[ch];
                const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
                const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
                strided_sum2(col, x, j0, j1, lane, 32, sa, sb);
            }
            sa = fsum_group<32>(sa);
            sb = fsum_group<32>(sb);
            if (lane == 0 && ch < L.chunks) {
                part_a[3 * ch] = (double)sa;  // exact for FP32 sums
                part_b[3 * ch] = (double)sb;
            }
        }
    }
}

// CHUNK rows of B's graph: each state's chunk partials merged as the
// one-state fixup merges them
__global__ void spmv_pair_fixup(SpmvLayout L, const int64_t* __restrict__ chunk_first,
                                const double* __restrict__ part_a, const double* __restrict__ part_b, double* P,
                                int64_t pstride, int level, int f32_from, float2* t_out, double alpha,
                                float alpha_f) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (u >= L.row_warp) return;
    const int64_t first = chunk_first[u], count = chunk_first[u + 1] - first;
    if (level < f32_from) {
        const XAcc ta = merge_chunks_warp(part_a, first, count);
        const XAcc tb = merge_chunks_warp(part_b, first, count);
        if ((threadIdx.x & 31) == 0) store_pair64((double2*)(P + (size_t)level * pstride), t_out, u, ta, tb, alpha);
    } else {
        const float ta = chunk_tree_warp(part_a, first, count);
        const float tb = chunk_tree_warp(part_b, first, count);
        if ((threadIdx.x & 31) == 0)
            ((float2*)(P + (size_t)level * pstride))[u] = make_float2(__fmul_rn(alpha_f, ta), __fmul_rn(alpha_f, tb));
    }
}

// Level 1 of both states: the degrees (A 1 = deg) in A's and in B's graph
template <typename OffA, typename OffB>
__global__ void pair_degree_kernel(const OffA* __restrict__ rp_a, const OffB* __restrict__ rp_b, int64_t n,
                                   double* P, int64_t pstride, float2* t_out, double alpha) {
    double2* y = (double2*)(P + (size_t)pstride);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const double a = __dmul_rn(alpha, (double)((int64_t)rp_a[u + 1] - (int64_t)rp_a[u]));
        const double b = __dmul_rn(alpha, (double)((int64_t)rp_b[u + 1] - (int64_t)rp_b[u]));
        y[u] = make_double2(a, b);
        if (t_out) t_out[u] = make_float2(f64_to_f32_rn(a), f64_to_f32_rn(b));
    }
}

// The rows the second batch changed (both endpoints of each update, internal
// ids): marked in vbits; the non-CHUNK ones listed (each once)
__global__ void pair_mark_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                 const int32_t* __restrict__ inv, int64_t row_warp, uint32_t* vbits,
                                 int32_t* rows, unsigned long long* nrows) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * m; e += stride) {
        const int32_t u = inv[(e & 1) ? dst[e >> 1] : src[e >> 1]];
        const uint32_t bit = 1u << (u & 31);
        const uint32_t old = atomicOr(&vbits[u >> 5], bit);
        if (!(old & bit) && (int64_t)u >= row_warp) rows[atomicAdd(nrows, 1ull)] = u;
    }
}

// A's entries of the listed non-CHUNK rows from A's adjacency: the lane
// partition of the one-state kernel for the row's mode, over the A entries
// (stride 2) of the interleaved level below
template <typename Off>
__global__ void pair_fix_rows_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col, SpmvLayout L,
                                     const int32_t* __restrict__ rows, const unsigned long long* nrows_ptr,
                                     double* P, int64_t pstride, int level, int f32_from,
                                     const float2* __restrict__ t_in, float2* t_out, double alpha, float alpha_f) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t nrows = (int64_t)*nrows_ptr;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; w < nrows; w += warps) {
        const int64_t u = rows[w];
        const int64_t a = rowptr[u], e = rowptr[u + 1];
        if (level >= f32_from) {
            const float* __restrict__ x = level == f32_from ? (const float*)t_in
                                                            : (const float*)(P + (size_t)(level - 1) * pstride);
            float s = 0.0f;
            if (u >= L.row_thread) {
                if (lane == 0) s = strided_sum<float, float, 2>(col, x, a, e, 0, 1);
            } else if (u >= L.row_octet) {
                if (lane < 8) s = strided_sum<float, float, 2>(col, x, a, e, lane, 8);
                s = fsum_group<8>(s);
            } else {
                s = strided_sum<float, float, 2>(col, x, a, e, lane, 32);
                s = fsum_group<32>(s);
            }
            if (lane == 0) ((float*)(P + (size_t)level * pstride))[2 * u] = __fmul_rn(alpha_f, s);
            continue;
        }
        const double* __restrict__ x = P + (size_t)(level - 1) * pstride;
        XAcc s = xacc_zero();
        if (u >= L.row_thread) {
            if (lane == 0) s = strided_xsum<4, 2>(col, x, a, e, 0, 1);
        } else if (u >= L.row_octet) {
            if (lane < 8) s = strided_xsum<4, 2>(col, x, a, e, lane, 8);
            s = xacc_group_sum<8>(s);
        } else {
            s = strided_xsum<8, 2>(col, x, a, e, lane, 32);
            s = xacc_group_sum<32>(s);
        }
        if (lane == 0) {
            const double sd = __dmul_rn(alpha, xacc_to_double(s));
            (P + (size_t)level * pstride)[2 * u] = sd;
            if (t_out) ((float*)t_out)[2 * u] = f64_to_f32_rn(sd);
        }
    }
}

// A's chunk partials of the marked CHUNK rows, with A's chunk table
template <typename Off>
__global__ void pair_fix_hub_chunks_kernel(const Off* __restrict__ rowptr, const int32_t* __restrict__ col,
                                           SpmvLayout L, const int32_t* __restrict__ chunk_row,
                                           const int64_t* __restrict__ chunk_first, double* part,
                                           const uint32_t* __restrict__ vbits, const double* P, int64_t pstride,
                                           int level, int f32_from, const float2* __restrict__ t_in) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; ch < L.chunks; ch += warps) {
        const int64_t u = chunk_row[ch];
        if (!visited(vbits, u)) continue;
        const int64_t j0 = (int64_t)rowptr[u] + (ch - chunk_first[u]) * (int64_t)CHUNK_ARCS;
        const int64_t j1 = min(j0 + (int64_t)CHUNK_ARCS, (int64_t)rowptr[u + 1]);
        if (level >= f32_from) {
            const float* __restrict__ x = level == f32_from ? (const float*)t_in
                                                            : (const float*)(P + (size_t)(level - 1) * pstride);
            const float s = fsum_group<32>(strided_sum<float, float, 2>(col, x, j0, j1, lane, 32));
            if (lane == 0) part[3 * ch] = (double)s;
        } else {
            const XAcc t = xacc_group_sum<32>(strided_xsum<8, 2>(col, P + (size_t)(level - 1) * pstride, j0, j1, lane, 32));
            if (lane == 0) store_part(part, ch, t);
        }
    }
}

// A's entries of the marked CHUNK rows: A's partials merged
__global__ void pair_fix_hub_rows_kernel(SpmvLayout L, const int64_t* __restrict__ chunk_first,
                                         const double* __restrict__ part, const uint32_t* __restrict__ vbits,
                                         double* P, int64_t pstride, int level, int f32_from, float2* t_out,
                                         double alpha, float alpha_f) {
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (u >= L.row_warp || !visited(vbits, u)) return;
    const int64_t first = chunk_first[u], count = chunk_first[u + 1] - first;
    if (level >= f32_from) {
        const float t = chunk_tree_warp(part, first, count);
        if ((threadIdx.x & 31) == 0) ((float*)(P + (size_t)level * pstride))[2 * u] = __fmul_rn(alpha_f, t);
        return;
    }
    const XAcc t = merge_chunks_warp(part, first, count);
    if ((threadIdx.x & 31) == 0) {
        const double sd = __dmul_rn(alpha, xacc_to_double(t));
        (P + (size_t)level * pstride)[2 * u] = sd;
        if (t_out) ((float*)t_out)[2 * u] = f64_to_f32_rn(sd);
    }
}

// state `st` (0: A, 1: B) of levels 1..r into the handle's walk slots, and of
// the FP32 roundings into s32
__global__ void pair_split_kernel(const double* __restrict__ P, int64_t pstride, int r, int f32_from, int st,
                                  double* walk, IterParams p, const float* __restrict__ t_pair, float* s32) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < p.n; u += stride) {
        for (int level = 1; level <= r; ++level) {
            const double* lv = P + (size_t)level * pstride;
            if (level < f32_from) walk_slot(walk, p, level)[u] = lv[2 * u + st];
            else ((float*)walk_slot(walk, p, level))[u] = ((const float*)lv)[2 * u + st];
        }
        if (s32) s32[u] = t_pair[2 * u + st];
    }
}

}  // namespace

// Levels 1..r of both states (see above).  ga: A's graph (current), gb: B's
// graph (the prepared spares, its own layout and chunk table); bsrc/bdst: the
// second batch (original ids), m of them; P: (r + 1) interleaved slots of
// pstride doubles; t_pair: n pairs of FP32 roundings (cert mode); part: 6 words
// per chunk of B's graph (A's partials, then B's); vbits/rows/nrows: scratch of
// the dynamic path (vbits and nrows cleared here).
cudaError_t launch_pair_levels(const DeviceGraph& ga, const DeviceGraph& gb, const int32_t* bsrc,
                               const int32_t* bdst, int64_t m, const IterParams& p, int r, int f32_from,
                               int t_level, double* P, int64_t pstride, float* t_pair, double* part,
                               uint32_t* vbits, int32_t* rows, unsigned long long* nrows, cudaStream_t st) {
    const int64_t n = ga.n;
    cudaError_t e = cudaMemsetAsync(vbits, 0, (size_t)((n + 31) / 32) * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(nrows, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (m > 0)
        pair_mark_kernel<<<(unsigned)std::min<int64_t>((2 * m + 255) / 256, 152 * 8), 256, 0, st>>>(
            bsrc, bdst, m, ga.inv, ga.layout.row_warp, vbits, rows, nrows);
    const int64_t blocks_n = std::min<int64_t>(std::max<int64_t>((n + BLOCK - 1) / BLOCK, 1), 152 * 8);
    float2* t2 = (float2*)t_pair;
    {
        float2* t_out = (p.cert && t_level == 1) ? t2 : nullptr;
#define KATZ_PAIR_DEG(OA, OB)                                                                          \
    pair_degree_kernel<OA, OB><<<(unsigned)blocks_n, BLOCK, 0, st>>>((const OA*)ga.rowptr, (const OB*)gb.rowptr, n, \
                                                                      P, pstride, t_out, p.alpha)
        if (ga.off64 && gb.off64) KATZ_PAIR_DEG(int64_t, int64_t);
        else if (ga.off64) KATZ_PAIR_DEG(int64_t, int32_t);
        else if (gb.off64) KATZ_PAIR_DEG(int32_t, int64_t);
        else KATZ_PAIR_DEG(int32_t, int32_t);
#undef KATZ_PAIR_DEG
    }
    const SpmvLayout& LB = gb.layout;
    const SpmvLayout& LA = ga.layout;
    double* part_a = part;
    double* part_b = part + 3 * std::max<int64_t>(LB.chunks, 1);
    for (int level = 2; level <= r; ++level) {
        float2* t_out = (p.cert && level == t_level) ? t2 : nullptr;
        if (LB.blocks_total > 0) {
            if (gb.off64)
                spmv_pair_kernel<int64_t><<<(unsigned)LB.blocks_total, BLOCK, 0, st>>>(
                    (const int64_t*)gb.rowptr, gb.col, LB, gb.chunk_row, gb.chunk_first, P, pstride, level, f32_from,
                    t2, t_out, part_a, part_b, p.alpha, p.alpha_f);
            else
                spmv_pair_kernel<int32_t><<<(unsigned)LB.blocks_total, BLOCK, 0, st>>>(
                    (const int32_t*)gb.rowptr, gb.col, LB, gb.chunk_row, gb.chunk_first, P, pstride, level, f32_from,
                    t2, t_out, part_a, part_b, p.alpha, p.alpha_f);
        }
        if (LB.row_warp > 0)
            spmv_pair_fixup<<<(unsigned)((LB.row_warp * 32 + 127) / 128), 128, 0, st>>>(
                LB, gb.chunk_first, part_a, part_b, P, pstride, level, f32_from, t_out, p.alpha, p.alpha_f);
        // A's entries of the rows the second batch changed, from A's rows
        if (m > 0) {
            const unsigned fb = (unsigned)std::min<int64_t>((2 * m + 7) / 8, 152 * 32);
            if (ga.off64)
                pair_fix_rows_kernel<int64_t><<<fb, 256, 0, st>>>((const int64_t*)ga.rowptr, ga.col, LA, rows, nrows,
                                                                 P, pstride, level, f32_from, t2, t_out, p.alpha,
                                                                 p.alpha_f);
            else
                pair_fix_rows_kernel<int32_t><<<fb, 256, 0, st>>>((const int32_t*)ga.rowptr, ga.col, LA, rows, nrows,
                                                                 P, pstride, level, f32_from, t2, t_out, p.alpha,
                                                                 p.alpha_f);
            if (LA.chunks > 0) {
                const unsigned cb = (unsigned)std::min<int64_t>((LA.chunks + 7) / 8, 152 * 32);
                if (ga.off64)
                    pair_fix_hub_chunks_kernel<int64_t><<<cb, 256, 0, st>>>(
                        (const int64_t*)ga.rowptr, ga.col, LA, ga.chunk_row, ga.chunk_first, ga.chunk_part, vbits, P,
                        pstride, level, f32_from, t2);
                else
                    pair_fix_hub_chunks_kernel<int32_t><<<cb, 256, 0, st>>>(
                        (const int32_t*)ga.rowptr, ga.col, LA, ga.chunk_row, ga.chunk_first, ga.chunk_part, vbits, P,
                        pstride, level, f32_from, t2);
                pair_fix_hub_rows_kernel<<<(unsigned)((LA.row_warp * 32 + 127) / 128), 128, 0, st>>>(
                    LA, ga.chunk_first, ga.chunk_part, vbits, P, pstride, level, f32_from, t_out, p.alpha, p.alpha_f);
            }
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_split(const DeviceGraph& g, const IterBuffers& b, const IterParams& p, int r, int f32_from,
                              int state, const double* P, int64_t pstride, const float* t_pair, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>(std::max<int64_t>((g.n + 255) / 256, 1), 152 * 8);
    pair_split_kernel<<<(unsigned)blocks, 256, 0, st>>>(P, pstride, r, f32_from, state, (double*)b.walk, p, t_pair,
                                                        p.cert ? b.s32 : nullptr);
    return cudaGetLastError();
}

// Block ranges of the four row modes from the internal row boundaries.
SpmvLayout make_layout(int64_t n, int64_t row_warp, int64_t row_octet, int64_t row_thread, int64_t chunks) {
    SpmvLayout L{};
    L.n = n;
    L.row_warp = row_warp;
    L.row_octet = row_octet;
    L.row_thread = row_thread;
    L.chunks = chunks;
    const int64_t bc = (chunks + WARPS - 1) / WARPS;
    const int64_t bw = (row_octet - row_warp + WARPS - 1) / WARPS;
    const int64_t bo = (row_thread - row_octet + BLOCK / 8 - 1) / (BLOCK / 8);
    const int64_t bt = (n - row_thread + BLOCK - 1) / BLOCK;
    L.blk_warp = bc;
    L.blk_octet = bc + bw;
    L.blk_thread = bc + bw + bo;
    L.blocks_total = bc + bw + bo + bt;
    return L;
}

}  // namespace katz
