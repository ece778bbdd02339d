// Emulated-FP64 complex GEMM on the tcgen05 tensor cores (the separator Schur updates and the
// selected-inverse products of the factor and selinv schedules).
//
// Method (an error-free splitting in the spirit of Ozaki, Ogita, Oishi and Rump's scheme, with
// BF16 digits and FP32 tensor-core accumulation):
//  * complex operands are stacked as real matrices: A'' = [Re A | Im A] (M x 2K) and, per
//    NC-column tile of B, NC rows [Re B | -Im B] followed by NC rows [Im B | Re B], so that one
//    real product gives Re C in the first NC accumulator columns and Im C in the next NC;
//  * every row of A'' (column of B) is scaled by a power of two 2^E with |x| < 2^E and written as
//    S balanced base-256 digits, x = 2^(E-7) sum_t d_t 2^(-8(t-1)), d_1 in [-128,128],
//    d_t in [-128,127]; digit t is stored pre-scaled, d_t 2^(-8(t-1)), exactly as BF16.  The
//    digits come from the FP64 bit pattern with integer operations only;
//  * the slice products A_t B_u^T with t+u <= S+1 are accumulated in TMEM, by default one
//    accumulator per scale t+u (S of them, 2NC columns each): the B digits of a stage are
//    consecutive rows of one K-major block, so A_t times [B_1; ...; B_{S+1-t}] is one wide MMA (or
//    two, N <= 256) whose output columns fall into the accumulators of t+1 .. S+1 - each operand
//    tile is read from shared memory once per digit instead of once per product, which keeps
//    the tensor pipe fed at N = 2NC = 80.  Within an accumulator every partial sum over a
//    256-element K chunk has at most four products per K for the leading four scales, so it is
//    an integer of at most 2^24 times a power of two and exact in FP32 (the lower scales, 2^-32
//    and below, may round at 2^-24 of themselves).  Every accumulator is read out after every
//    chunk into a per-element float-float (hi, lo) sum.  The optional tail variants keep t+u = 2
//    .. BANDS in their own accumulators and the rest in a shared tail, where the tensor core
//    drops the low bits of the smaller products: BANDS = 5 (NC = 48) gives a floor near 2^-43 of
//    the result, BANDS = 4 (NC = 64) near 2^-38;
//  * the epilogue scales by 2^(E_m + F_n - 14) and forms C = alpha*(hi+lo)*scale + beta*C.
// Pipeline (persistent, one CTA per SM, tiles claimed from a counter in list order and handed on
// through a small shared-memory queue): warp 0 claims tiles and issues TMA loads (2 to 6 stages,
// as many as fit shared memory, of S A tiles 128x32 and S B tiles 2NCx32, BF16, 64-byte
// swizzle), one thread of warp 1 issues the MMAs (M=128, K=16), warps 2-17 read TMEM and convert
// and store finished tiles while the next tile's MMAs run.  Every mbarrier wait is bounded: on
// time-out the kernel flags NDSI timeout status, drains what it issued and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdint>

#include "kernels.cuh"
#include "split_gemm.cuh"

namespace ndsi {

void build_split_schedule(const Plan& P, int slices, const std::vector<int8_t>& bands,
                          std::vector<SplitItem>& items, std::vector<SplitStep>& steps,
                          std::vector<GemmTile>& tiles, std::vector<SliceBlock>& blocks) {
    items.assign(P.gemm_items.size(), SplitItem{});
    steps.clear();
    tiles.clear();
    blocks.clear();
    for (size_t li = 0; li < P.launches.size(); ++li) {
        const Launch& l = P.launches[li];
        if (!split_eligible(l)) continue;
        const int32_t nc = split_nc(slices, bands[li]);
        SplitStep st{};
        st.nc = nc;
        int32_t kmax = 0;
        st.tfirst = static_cast<int64_t>(tiles.size());
        st.sa_first = static_cast<int64_t>(blocks.size());
        for (int64_t i = 0; i < l.count; ++i) {
            const GemmItem& g = P.gemm_items[l.first + i];
            SplitItem& s = items[l.first + i];
            s.Mpad = (g.M + kSplitBM - 1) / kSplitBM * kSplitBM;
            s.Npad = (g.N + nc - 1) / nc * nc;
            s.Kpad = (g.K + kSplitKB - 1) / kSplitKB * kSplitKB;
            s.rowA = st.rowsA;
            s.rowB = st.rowsB;
            s.erowA = st.erowsA;
            s.erowB = st.erowsB;
            st.rowsA += static_cast<int64_t>(slices) * s.Mpad;
            st.rowsB += static_cast<int64_t>(slices) * 2 * s.Npad;
            st.erowsA += s.Mpad;
            st.erowsB += s.Npad;
            kmax = std::max(kmax, s.Kpad);
            // Tile order.  The persistent CTAs take consecutive tiles, about kSplitConcurrentTiles
            // at a time, and move through K at about the same pace, so a K-block of an operand tile
            // that several running CTAs share is read from HBM once and from L2 by the others.
            // Tiles are ordered in groups of g row tiles (column tiles) swept across all column
            // (row) tiles; the group keeps its operand in L2 for the whole sweep when it fits a
            // share of L2, and otherwise shares it only among the tiles running together.  The
            // group size and direction with the fewest estimated DRAM bytes win: a wide operand
            // streamed once per 128-row block (row-block order) read a 4000-wide L_RJ 9x over.
            const int32_t mt = (g.M + kSplitBM - 1) / kSplitBM, nt = (g.N + nc - 1) / nc;
            const double a_tile = static_cast<double>(slices) * 2.0 * s.Kpad * 2.0 * kSplitBM;
            const double b_tile = static_cast<double>(slices) * 2.0 * s.Kpad * 2.0 * 2.0 * nc;
            // DRAM bytes of the order "groups of gp tiles along P swept across all q of Q"
            auto traffic = [&](int32_t gp, int32_t np_, int32_t nq, double p_tile, double q_tile) {
                const double groups = std::ceil(static_cast<double>(np_) / gp);
                const double q_bytes = q_tile * nq * groups;      // each q tile once per group
                double p_reads = 1.0;                             // the group's p tiles...
                if (gp * p_tile > kSplitL2Share) {                // ...unless they leave L2
                    const double together = std::max(1.0, static_cast<double>(kSplitConcurrentTiles) / gp);
                    p_reads = std::ceil(nq / together);
                }
                return q_bytes + p_tile * np_ * p_reads;
            };
            int32_t best_g = 1;
            bool rows_grouped = true;
            double best = -1.0;
            for (int32_t gsz = 1; gsz <= mt; ++gsz) {
                const double t = traffic(gsz, mt, nt, a_tile, b_tile);
                if (best < 0 || t < best) { best = t; best_g = gsz; rows_grouped = true; }
            }
            for (int32_t gsz = 1; gsz <= nt; ++gsz) {
                const double t = traffic(gsz, nt, mt, b_tile, a_tile);
                if (t < best) { best = t; best_g = gsz; rows_grouped = false; }
            }
            auto push = [&](int32_t mi, int32_t ni) {
                const int32_t m0 = mi * kSplitBM, n0 = ni * nc;
                if (l.lower && n0 > m0 + kSplitBM - 1) return;
                tiles.push_back(GemmTile{static_cast<int32_t>(i), m0, n0, 0});
            };
            if (rows_grouped) {
                for (int32_t m1 = 0; m1 < mt; m1 += best_g)
                    for (int32_t ni = 0; ni < nt; ++ni)
                        for (int32_t mi = m1; mi < std::min(mt, m1 + best_g); ++mi) push(mi, ni);
            } else {
                for (int32_t n1 = 0; n1 < nt; n1 += best_g)
                    for (int32_t mi = 0; mi < mt; ++mi)
                        for (int32_t ni = n1; ni < std::min(nt, n1 + best_g); ++ni) push(mi, ni);
            }
        }
        st.tcount = static_cast<int64_t>(tiles.size()) - st.tfirst;
        // slicing: one pass over the operand when a block of rows x K fits the shared-memory
        // budget (32, 16, 8 or 4 rows), else two passes over 32-row blocks
        int32_t kreal = 0;
        for (int64_t i = 0; i < l.count; ++i) kreal = std::max(kreal, P.gemm_items[l.first + i].K);
        st.slice_ldt = kreal + 1;
        st.slice_rows = 32;
        while (st.slice_rows > 4 && static_cast<int64_t>(st.slice_rows) * st.slice_ldt * 16 > kSplitSlice1Smem)
            st.slice_rows /= 2;
        if (static_cast<int64_t>(st.slice_rows) * st.slice_ldt * 16 > kSplitSlice1Smem) {
            // very long rows: one or two rows per block with a larger shared-memory allocation
            st.slice_rows = 2;
            if (static_cast<int64_t>(st.slice_rows) * st.slice_ldt * 16 > kSplitSlice1SmemWide) st.slice_rows = 1;
            if (static_cast<int64_t>(st.slice_rows) * st.slice_ldt * 16 > kSplitSlice1SmemWide) {
                st.slice_rows = kSplitSliceRows;
                st.slice_ldt = 0;
            }
        }
        for (int64_t i = 0; i < l.count; ++i) {
            const GemmItem& g = P.gemm_items[l.first + i];
            for (int32_t r0 = 0; r0 < g.M; r0 += st.slice_rows) blocks.push_back(SliceBlock{static_cast<int32_t>(i), r0});
        }
        st.sa_count = static_cast<int64_t>(blocks.size()) - st.sa_first;
        st.sb_first = static_cast<int64_t>(blocks.size());
        for (int64_t i = 0; i < l.count; ++i) {
            const GemmItem& g = P.gemm_items[l.first + i];
            for (int32_t n0 = 0; n0 < g.N; n0 += st.slice_rows) blocks.push_back(SliceBlock{static_cast<int32_t>(i), n0});
        }
        st.sb_count = static_cast<int64_t>(blocks.size()) - st.sb_first;
        st.Kcols = std::max(64, 2 * kmax);
        st.Kcols = (st.Kcols + 63) / 64 * 64;
        steps.push_back(st);
    }
}

namespace {

// ------------------------------------------------------------------------------------ PTX ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Wait for the given phase parity; gives up (raising *abort) after kWaitLimitNs or when another
// role already aborted.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (*abort) return false;
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) {
            *abort = 1;
            return false;
        }
    }
}
// Bounded wait used while draining after an abort (ignores the abort flag).
__device__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM loads without the wait: the registers are valid only after tmem_wait_ld, which names them
// as outputs so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld4_async(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld2_async(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
}
// W consecutive accumulator columns (W even) of this warp's 32 lanes into r[0, W)
template <int W>
__device__ __forceinline__ void tmem_ld_cols_async(uint32_t taddr, uint32_t* r) {
#pragma unroll
    for (int j0 = 0; j0 + 8 <= W; j0 += 8) tmem_ld8_async(taddr + j0, r + j0);
    if constexpr (W % 8 >= 4) tmem_ld4_async(taddr + (W / 8) * 8, r + (W / 8) * 8);
    if constexpr (W % 4 == 2) tmem_ld2_async(taddr + (W / 4) * 4, r + (W / 4) * 4);
}
template <int N>
__device__ __forceinline__ void tmem_wait_ld(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}

// Bytes of one K-major tile row (the stage's K in BF16) and the matching swizzle.
constexpr int kRowBytes = kSplitKB * 2;
constexpr int kK16Steps = kSplitKB / 16;  // K16 MMA steps per stage
// Shared-memory matrix descriptor: K-major tile of 8-row x kRowBytes swizzle atoms stacked along M
// (stride 8 rows), descriptor version 1, 32-byte (layout 6) or 64-byte (layout 4) swizzle.
__device__ __forceinline__ uint64_t sdesc_sw(uint32_t saddr) {
    uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1) << 16;
    d |= static_cast<uint64_t>((8 * kRowBytes) >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(kRowBytes == 32 ? 6 : 4) << 61;
    return d;
}
// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = n (multiple of 16).
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// float-float accumulation hi + lo += v (Knuth's two-sum).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += e;
}

// (hi + lo) * 2^e rounded to nearest double, using integer operations only (GB300's FP64 pipe is
// the scarce unit): both floats become signed integer mantissas at a common exponent, their
// exact sum (an int64) is rounded to 53 bits and packed with the combined exponent.  Out of the
// normal double range it falls back to FP64 arithmetic.
// Out-of-range results (never produced by finite fronts in practice) take the FP64 route in a
// separate function so that the common path carries no FP64 instructions, even predicated ones.
__device__ __noinline__ double ff_to_double_slow(float hi, float lo, int e, bool negate) {
    const double v = ldexp(static_cast<double>(hi) + static_cast<double>(lo), e);
    return negate ? -v : v;
}

__device__ __forceinline__ double ff_to_double_scaled(float hi, float lo, int e, bool negate = false) {
    const uint32_t bh = __float_as_uint(hi), bl = __float_as_uint(lo);
    const int eh = static_cast<int>((bh >> 23) & 0xFF), el = static_cast<int>((bl >> 23) & 0xFF);
    int64_t mh = eh ? static_cast<int64_t>((bh & 0x7FFFFFu) | 0x800000u) : 0;
    int64_t ml = el ? static_cast<int64_t>((bl & 0x7FFFFFu) | 0x800000u) : 0;
    if (bh >> 31) mh = -mh;
    if (bl >> 31) ml = -ml;
    int64_t S;
    int E0;
    if (ml == 0) {
        if (mh == 0) return 0.0;
        S = mh;
        E0 = eh - 150;
    } else if (mh == 0) {
        S = ml;
        E0 = el - 150;
    } else {
        int64_t big = mh, small = ml;
        int ebig = eh, esmall = el;
        if (el > eh) {
            big = ml;
            small = mh;
            ebig = el;
            esmall = eh;
        }
        const int d = ebig - esmall;
        if (d <= 38) {
            S = (big << d) + small;
            E0 = esmall - 150;
        } else {
            S = (big << 38) + (small >> (d - 38));
            E0 = ebig - 150 - 38;
        }
    }
    const bool neg = (S < 0) != negate;
    uint64_t u = static_cast<uint64_t>(S < 0 ? -S : S);
    if (u == 0) return 0.0;
    const int nbits = 64 - __clzll(static_cast<long long>(u));
    int exp2;
    uint64_t mant;
    if (nbits > 53) {
        int sh = nbits - 53;
        mant = u >> sh;
        const uint64_t rem = u & ((uint64_t(1) << sh) - 1);
        const uint64_t half = uint64_t(1) << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) ++mant;
        if (mant >> 53) {
            mant >>= 1;
            ++sh;
        }
        exp2 = E0 + e + sh + 52;
    } else {
        mant = u << (53 - nbits);
        exp2 = E0 + e - (53 - nbits) + 52;
    }
    const int biased = exp2 + 1023;
    if (biased <= 0 || biased >= 2047) return ff_to_double_slow(hi, lo, e, negate);
    const uint64_t bits = (static_cast<uint64_t>(neg) << 63) | (static_cast<uint64_t>(biased) << 52) |
                          (mant & ((uint64_t(1) << 52) - 1));
    return __longlong_as_double(static_cast<long long>(bits));
}

// ----------------------------------------------------------------------------- slicing -----
// Biased FP64 exponent of x with zero mapped to -1 (and subnormals to 1).
__device__ __forceinline__ int fp64_expo(double x) {
    const int64_t b = __double_as_longlong(x);
    const int ex = static_cast<int>((b >> 52) & 0x7FF);
    if ((b & 0x7FFFFFFFFFFFFFFFLL) == 0) return -1;
    return ex == 0 ? 1 : ex;
}

// Balanced base-256 digits of x / 2^(E+1) * 2^(8S): d[0] in [-128,128], d[1..S-1] in [-128,127].
template <int S>
__device__ __forceinline__ void fp64_digits(double x, int E, int* d) {
    const int64_t b = __double_as_longlong(x);
    int ex = static_cast<int>((b >> 52) & 0x7FF);
    int64_t mant = b & 0xFFFFFFFFFFFFFLL;
    if (ex) mant |= 0x10000000000000LL; else ex = 1;
    const int shift = ex - 1076 - E + 8 * S;
    int64_t F;
    if (shift >= 0) {
        F = mant << shift;
    } else {
        const int rsh = -shift;
        F = rsh >= 62 ? 0 : (((mant >> (rsh - 1)) + 1) >> 1);
    }
    if (b < 0) F = -F;
#pragma unroll
    for (int t = S - 1; t >= 1; --t) {
        int low = static_cast<int>(F & 0xFF);
        if (low >= 128) low -= 256;
        d[t] = low;
        F = (F - low) >> 8;
    }
    d[0] = static_cast<int>(F);
}

// Same digits with 32-bit integer work: the fixed-point value is split into 24-bit halves
// (S <= 6: F < 2^47), the low half's balanced digits carry into the high half.
template <int S>
__device__ __forceinline__ void fp64_digits32(double x, int E, int* d) {
    if (S > 6) {
        fp64_digits<S>(x, E, d);
        return;
    }
    const int64_t b = __double_as_longlong(x);
    int ex = static_cast<int>((b >> 52) & 0x7FF);
    int64_t mant = b & 0xFFFFFFFFFFFFFLL;
    if (ex) mant |= 0x10000000000000LL; else ex = 1;
    const int rsh = 1076 + E - 8 * S - ex;  // >= 6 for S <= 6
    const uint64_t F = rsh >= 62 ? 0 : (((static_cast<uint64_t>(mant) >> (rsh - 1)) + 1) >> 1);
    int lo = static_cast<int>(F & 0xFFFFFF);
    int hi = static_cast<int>(F >> 24);
    const bool neg = b < 0;
    if (neg) {
        // -(hi*2^24 + lo) = (-hi-1)*2^24 + (2^24 - lo), keeping lo in [0, 2^24)
        if (lo) {
            hi = -hi - 1;
            lo = 0x1000000 - lo;
        } else {
            hi = -hi;
        }
    }
    // digits S-1 .. S-3 from lo (0-based index), the rest from hi
#pragma unroll
    for (int t = S - 1; t >= 1; --t) {
        int& v = (t >= S - 3) ? lo : hi;
        int low = v & 0xFF;
        if (low >= 128) low -= 256;
        d[t] = low;
        v = (v - low) >> 8;
        if (t == S - 3) hi += lo;  // carry out of the low half
    }
    d[0] = hi;
}

// d * 2^(-8t) as an exact FP32 value, |d| <= 128: 1.5*2^23 + d has ulp 1, so adding d to its bit
// pattern and subtracting 1.5*2^23 gives d exactly; the power-of-two scale is exact too.  With at
// most 8 significant bits the value's BF16 pattern is the upper half of the FP32 pattern.
__device__ __forceinline__ uint32_t digit_f32_bits(int d, int t) {
    const float f = (__int_as_float(0x4B400000 + d) - 12582912.0f) * __int_as_float((127 - 8 * t) << 23);
    return __float_as_uint(f);
}
// Two digits as a packed BF16 pair (first in the low half).
__device__ __forceinline__ uint32_t bf16_pair(int d0, int d1, int t) {
    return __byte_perm(digit_f32_bits(d0, t), digit_f32_bits(d1, t), 0x7632);
}

// x / 2^(E+1) * 2^(8S), rounded to the nearest integer, in two's complement (S <= 6: the shift
// is at least 6 bits to the right, see fp64_digits32).
template <int S>
__device__ __forceinline__ int64_t fp64_scaled(double x, int E) {
    const int64_t b = __double_as_longlong(x);
    int ex = static_cast<int>((b >> 52) & 0x7FF);
    int64_t mant = b & 0xFFFFFFFFFFFFFLL;
    if (ex) mant |= 0x10000000000000LL; else ex = 1;
    const int rsh = 1076 + E - 8 * S - ex;
    const int64_t mag = rsh >= 62 ? 0 : static_cast<int64_t>(((static_cast<uint64_t>(mant) >> (rsh - 1)) + 1) >> 1);
    return b < 0 ? -mag : mag;
}

// Packed BF16 pairs w[t] = (digit t of x0 | digit t of x1 << 16), digit t scaled by 2^(-8t): the
// same balanced base-256 digits as fp64_digits32.  Adding 128 to every digit below the top one
// turns the balanced digits into the plain bytes of the sum (carries included), so each digit is
// one byte extract and the exact FP32 conversion of digit_f32_bits with the bias folded in.
template <int S>
__device__ __forceinline__ void slice_pair(double x0, double x1, int E, uint32_t* w) {
    if (S > 6) {
        int d0[S], d1[S];
        fp64_digits32<S>(x0, E, d0);
        fp64_digits32<S>(x1, E, d1);
#pragma unroll
        for (int t = 0; t < S; ++t) w[t] = bf16_pair(d0[t], d1[t], t);
        return;
    }
    int64_t bias = 0;
#pragma unroll
    for (int t = 0; t < S - 1; ++t) bias |= static_cast<int64_t>(128) << (8 * t);
    const int64_t g0 = fp64_scaled<S>(x0, E) + bias, g1 = fp64_scaled<S>(x1, E) + bias;
    const uint32_t lo0 = static_cast<uint32_t>(g0), hi0 = static_cast<uint32_t>(static_cast<uint64_t>(g0) >> 32);
    const uint32_t lo1 = static_cast<uint32_t>(g1), hi1 = static_cast<uint32_t>(static_cast<uint64_t>(g1) >> 32);
#pragma unroll
    for (int t = 1; t < S; ++t) {
        const int k = S - 1 - t;  // byte of the biased sum holding digit t
        // one byte permute builds the FP32 bits 0x4B4000bb (= 2^23 + 2^22 + b) from byte b, and one
        // FFMA gives (2^23 + 2^22 + b) 2^(-8t) - (2^23 + 2^22 + 128) 2^(-8t) = (b - 128) 2^(-8t):
        // every intermediate is exact
        const uint32_t sel = 0x7640u + static_cast<uint32_t>(k & 3);
        const uint32_t m0 = __byte_perm(k < 4 ? lo0 : hi0, 0x4B400000u, sel);
        const uint32_t m1 = __byte_perm(k < 4 ? lo1 : hi1, 0x4B400000u, sel);
        const float sc = __int_as_float((127 - 8 * t) << 23);
        const float f0 = fmaf(__uint_as_float(m0), sc, -12583040.0f * sc);
        const float f1 = fmaf(__uint_as_float(m1), sc, -12583040.0f * sc);
        w[t] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
    }
    const int t0 = static_cast<int>(g0 >> (8 * (S - 1))), t1 = static_cast<int>(g1 >> (8 * (S - 1)));
    w[0] = __byte_perm(__float_as_uint(__int_as_float(0x4B400000 + t0) - 12582912.0f),
                       __float_as_uint(__int_as_float(0x4B400000 + t1) - 12582912.0f), 0x7632);
}


struct SliceArgs {
    const GemmItem* items;
    const SplitItem* sitems;
    const SliceBlock* blocks;
    int64_t bfirst, ifirst;
    const double2* X;
    int64_t sX;
    int op;       // OP_N / OP_T / OP_S of the GEMM operand
    int isB;
    uint16_t* out;
    int64_t rows_pole;
    int32_t Kcols;
    int32_t* expo;
    int64_t erows_pole;
    int rows, ldt;  // one-pass slicer: rows per block and shared-memory row stride
    int nc;         // complex columns per output tile (B slices: groups of nc [Re|-Im], nc [Im|Re])
};

// Slices of one block of kSplitSliceRows rows of the stacked operand (A: rows m of op(A); B:
// columns n of op(B)).  A rows x 64-k complex tile is staged in shared memory with loads coalesced
// along whichever index is contiguous in memory.  Pass 1 finds the row exponents; pass 2 reads
// the rows again and turns two consecutive k per thread into digits, 32 threads per row, so every
// 4-byte store instruction of a warp fills one whole 128-byte line of a slice.  Blocks are few
// rows high so that the rows pass 1 read are still in L2 when pass 2 reads them.
constexpr int kSliceRows = kSplitSliceRows;
constexpr int kSliceK = 64;
constexpr int kSliceTPR = 256 / kSliceRows;  // pass-1 threads per row

template <int S>
__global__ void __launch_bounds__(256, 3) k_slice(const SliceArgs p) {
    __shared__ double2 tile[kSliceRows][kSliceK + 1];
    __shared__ int rowmax[kSliceRows];
    const SliceBlock blk = p.blocks[p.bfirst + blockIdx.x];
    const GemmItem it = p.items[p.ifirst + blk.item];
    const SplitItem si = p.sitems[p.ifirst + blk.item];
    const int64_t pole = blockIdx.y;
    const int nrows = p.isB ? it.N : it.M;
    const int K = it.K;
    const double2* base = p.X + pole * p.sX + (p.isB ? it.b_off : it.a_off);
    const int ld = p.isB ? it.ldb : it.lda;
    const bool sym = p.op == OP_S;
    const bool rows_contig = !sym && (p.isB ? p.op == OP_T : p.op == OP_N);
    const int tid = threadIdx.x;
    const int r = tid / kSliceTPR, kg = tid % kSliceTPR;
    const int row = blk.r0 + r;
    if (tid < kSliceRows) rowmax[tid] = -1;
    auto load_tile = [&](int k0) {
#pragma unroll
        for (int u = 0; u < kSliceRows * kSliceK / 256; ++u) {
            const int e = tid + 256 * u;
            int rr, kk;
            if (rows_contig) {
                rr = e % kSliceRows;
                kk = e / kSliceRows;
            } else {
                kk = e % kSliceK;
                rr = e / kSliceK;
            }
            const int gr = blk.r0 + rr, k = k0 + kk;
            double2 x = make_double2(0.0, 0.0);
            if (gr < nrows && k < K) {
                if (sym) {
                    const int hi = gr > k ? gr : k, lo = gr > k ? k : gr;
                    x = base[hi + static_cast<int64_t>(lo) * ld];
                } else if (rows_contig) {
                    x = base[gr + static_cast<int64_t>(k) * ld];
                } else {
                    x = base[k + static_cast<int64_t>(gr) * ld];
                }
            }
            tile[rr][kk] = x;
        }
    };
    __syncthreads();
    int lmax = -1;
    for (int k0 = 0; k0 < K; k0 += kSliceK) {
        load_tile(k0);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSliceK / kSliceTPR; ++j) {
            const double2 v = tile[r][kg * (kSliceK / kSliceTPR) + j];
            lmax = max(lmax, max(fp64_expo(v.x), fp64_expo(v.y)));
        }
        __syncthreads();
    }
    atomicMax(&rowmax[r], lmax);
    __syncthreads();
    const bool live = row < nrows;
    const int E = rowmax[r] < 0 ? -1021 : rowmax[r] - 1022;
    for (int k0 = 0; k0 < si.Kpad; k0 += kSliceK) {
        load_tile(k0);
        __syncthreads();
        // 32 threads per row, two consecutive k each: one 128-byte line per warp store
        const int kk = (tid % 32) * 2;
        const int col = k0 + kk;
#pragma unroll 1
        for (int pass = 0; pass < kSliceRows / 8; ++pass) {
            const int rr = pass * 8 + tid / 32;
            const int grow = blk.r0 + rr;
            if (grow >= nrows || col >= si.Kpad) continue;
            const int Er = rowmax[rr] < 0 ? -1021 : rowmax[rr] - 1022;
            int64_t o0, ost;
            if (!p.isB) {
                o0 = pole * p.rows_pole + si.rowA + grow;
                ost = si.Mpad;
            } else {
                o0 = pole * p.rows_pole + si.rowB + (grow / p.nc) * (2 * p.nc) + (grow % p.nc);
                ost = 2 * si.Npad;
            }
            const double2 v0 = tile[rr][kk];
            const double2 v1 = tile[rr][kk + 1];
            uint32_t wre[S], wim[S];
            slice_pair<S>(v0.x, v1.x, Er, wre);
            slice_pair<S>(v0.y, v1.y, Er, wim);
#pragma unroll
            for (int t = 0; t < S; ++t) {
                uint16_t* o1 = p.out + (o0 + t * ost) * p.Kcols;
                if (!p.isB) {
                    *reinterpret_cast<uint32_t*>(o1 + col) = wre[t];
                    *reinterpret_cast<uint32_t*>(o1 + si.Kpad + col) = wim[t];
                } else {
                    // rows [Re | -Im] and [Im | Re]; negation flips the BF16 sign bits
                    uint16_t* o2 = o1 + p.nc * static_cast<int64_t>(p.Kcols);
                    *reinterpret_cast<uint32_t*>(o1 + col) = wre[t];
                    *reinterpret_cast<uint32_t*>(o1 + si.Kpad + col) = wim[t] ^ 0x80008000u;
                    *reinterpret_cast<uint32_t*>(o2 + col) = wim[t];
                    *reinterpret_cast<uint32_t*>(o2 + si.Kpad + col) = wre[t];
                }
            }
        }
        __syncthreads();
    }
    if (live && kg == 0) p.expo[pole * p.erows_pole + (p.isB ? si.erowB : si.erowA) + row] = E;
}

// One-pass slicing: a block of `rows` (32, 16, 8, 4, or 2 or 1 for very long rows) operand rows
// with all K of them resident in shared memory, so every FP64 element is read from HBM once.  Loads are coalesced along the
// contiguous index; the row maxima come from rows-many thread groups; the digits are written by
// 32 threads per row with two consecutive k each, one 128-byte line per warp store.
template <int S>
__global__ void __launch_bounds__(256) k_slice1(const SliceArgs p) {
    extern __shared__ double2 t1[];  // [rows][ldt]
    __shared__ int rowmax[32];
    const SliceBlock blk = p.blocks[p.bfirst + blockIdx.x];
    const GemmItem it = p.items[p.ifirst + blk.item];
    const SplitItem si = p.sitems[p.ifirst + blk.item];
    const int64_t pole = blockIdx.y;
    const int nrows = p.isB ? it.N : it.M;
    const int K = it.K;
    const int R = p.rows, ldt = p.ldt;
    const double2* base = p.X + pole * p.sX + (p.isB ? it.b_off : it.a_off);
    const int ld = p.isB ? it.ldb : it.lda;
    const bool sym = p.op == OP_S;
    const bool rows_contig = !sym && (p.isB ? p.op == OP_T : p.op == OP_N);
    const int tid = threadIdx.x;
    if (tid < 32) rowmax[tid] = -1;
    // stage the rows with asynchronous 16-byte copies, all of a thread's copies in flight at once
    // (rows beyond the operand are zero-filled)
    const int total = R * K;
    for (int e = tid; e < total; e += 256) {
        int rr, kk;
        if (rows_contig) {
            rr = e % R;
            kk = e / R;
        } else {
            kk = e % K;
            rr = e / K;
        }
        const int gr = blk.r0 + rr;
        const double2* src = base;
        if (gr < nrows) {
            if (sym) {
                const int hi = gr > kk ? gr : kk, lo = gr > kk ? kk : gr;
                src = base + hi + static_cast<int64_t>(lo) * ld;
            } else if (rows_contig) {
                src = base + gr + static_cast<int64_t>(kk) * ld;
            } else {
                src = base + kk + static_cast<int64_t>(gr) * ld;
            }
        }
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(t1 + rr * ldt + kk));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                     "r"(gr < nrows ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    {
        const int tpr = 256 / R;  // threads per row
        const int rr = tid / tpr, kg = tid % tpr;
        int lmax = -1;
        for (int kk = kg; kk < K; kk += tpr) {
            const double2 v = t1[rr * ldt + kk];
            lmax = max(lmax, max(fp64_expo(v.x), fp64_expo(v.y)));
        }
        atomicMax(&rowmax[rr], lmax);
    }
    __syncthreads();
    const int half = si.Kpad / 2;  // k pairs per row
    for (int idx = tid; idx < R * half; idx += 256) {
        const int rr = idx / half, kk = 2 * (idx % half);
        const int grow = blk.r0 + rr;
        if (grow >= nrows) continue;
        const int Er = rowmax[rr] < 0 ? -1021 : rowmax[rr] - 1022;
        int64_t o0, ost;
        if (!p.isB) {
            o0 = pole * p.rows_pole + si.rowA + grow;
            ost = si.Mpad;
        } else {
            o0 = pole * p.rows_pole + si.rowB + (grow / p.nc) * (2 * p.nc) + (grow % p.nc);
            ost = 2 * si.Npad;
        }
        const double2 v0 = kk < K ? t1[rr * ldt + kk] : make_double2(0.0, 0.0);
        const double2 v1 = kk + 1 < K ? t1[rr * ldt + kk + 1] : make_double2(0.0, 0.0);
        uint32_t wre[S], wim[S];
        slice_pair<S>(v0.x, v1.x, Er, wre);
        slice_pair<S>(v0.y, v1.y, Er, wim);
#pragma unroll
        for (int t = 0; t < S; ++t) {
            uint16_t* o1 = p.out + (o0 + t * ost) * p.Kcols;
            if (!p.isB) {
                *reinterpret_cast<uint32_t*>(o1 + kk) = wre[t];
                *reinterpret_cast<uint32_t*>(o1 + si.Kpad + kk) = wim[t];
            } else {
                // rows [Re | -Im] and [Im | Re]; negation flips the BF16 sign bits
                uint16_t* o2 = o1 + p.nc * static_cast<int64_t>(p.Kcols);
                *reinterpret_cast<uint32_t*>(o1 + kk) = wre[t];
                *reinterpret_cast<uint32_t*>(o1 + si.Kpad + kk) = wim[t] ^ 0x80008000u;
                *reinterpret_cast<uint32_t*>(o2 + kk) = wim[t];
                *reinterpret_cast<uint32_t*>(o2 + si.Kpad + kk) = wre[t];
            }
        }
    }
    if (tid < R && blk.r0 + tid < nrows) {
        const int E = rowmax[tid] < 0 ? -1021 : rowmax[tid] - 1022;
        p.expo[pole * p.erows_pole + (p.isB ? si.erowB : si.erowA) + blk.r0 + tid] = E;
    }
}

// ---------------------------------------------------------------------------- the GEMM -----
struct GemmArgs {
    const GemmItem* items;
    const SplitItem* sitems;
    const GemmTile* tiles;
    int64_t tfirst, ifirst;
    int64_t rowsA, rowsB, erowsA, erowsB;
    const int32_t* expA;
    const int32_t* expB;
    double2* C;
    int64_t sC;
    int neg_alpha, add_c;  // alpha = -1 / +1; beta = 1 / 0
    int lower;
    int* status;
    int64_t tcount;        // tiles per pole
    int np;                // poles
};

constexpr int kTileBytes = kSplitBM * kRowBytes;  // 128 rows x kRowBytes
constexpr int kThreads = 576;
constexpr int kEpiWarps = 16;
constexpr int kTileQueue = 4;  // tiles claimed ahead of the epilogue

// OR of a predicate over the epilogue threads (named barrier 1), so that they all take the same
// branch.
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "n"(kEpiWarps * 32)
        : "memory");
    return r != 0;
}
// Epilogue TMEM read-out with two band buffers (register budget: 2 x 2CW values beside the 4CW
// float-float sums)
template <int CW>
constexpr bool kEpiDoubleBuffer = CW <= 12;

template <int NC>
__host__ __device__ constexpr int tile_bytes_b() { return 2 * NC * kRowBytes; }  // 2NC rows x kRowBytes
template <int S, int NC>
__host__ __device__ constexpr int stage_bytes() { return S * (kTileBytes + tile_bytes_b<NC>()); }
// barriers (256 B), the tile's row / column exponents (768 B) and up to 1 KB lost to aligning the
// tiles to 1024 bytes
constexpr int kSplitSmemExtra = 256 + 768 + 1024;
constexpr int kSplitMaxStages = 6;
// Pipeline depth: as many stages (2..6) as fit the 227 KB of shared memory a CTA may use.
template <int S, int NC>
__host__ __device__ constexpr int split_stages() {
    return (227 * 1024 - kSplitSmemExtra) / stage_bytes<S, NC>() >= kSplitMaxStages
               ? kSplitMaxStages
               : ((227 * 1024 - kSplitSmemExtra) / stage_bytes<S, NC>() < 2
                      ? 2
                      : (227 * 1024 - kSplitSmemExtra) / stage_bytes<S, NC>());
}
template <int S, int NC>
__host__ __device__ constexpr int split_smem_bytes() {
    return split_stages<S, NC>() * stage_bytes<S, NC>() + kSplitSmemExtra;
}
// Per-scale mode: one accumulator per t+u (any tile width other than the two tail variants).
template <int NC>
__host__ __device__ constexpr bool split_exact_mode() { return NC != kSplitBNc && NC != kSplitBNc5; }

// The MMAs of one A digit t in per-scale mode: A_t times the stage's B digits 0 .. S-1-t, which
// are consecutive rows of one K-major block, land in accumulator columns t*NB .. S*NB, i.e. the
// product with B_u in the accumulator of scale t+u.  Issued in pieces of at most 256 rows.
template <int S, int NB, int T, int R0>
__device__ __forceinline__ void issue_digit(uint32_t tmem, uint64_t da, uint64_t db0, int ks, uint32_t acc) {
    constexpr int rows = (S - T) * NB;
    if constexpr (R0 < rows) {
        constexpr int n = rows - R0 < 256 ? rows - R0 : 256;
        const uint64_t db = db0 + static_cast<uint64_t>((R0 * kRowBytes + ks * 32) >> 4);
        umma_bf16(tmem + T * NB + R0, da, db, idesc_bf16(n), acc);
        issue_digit<S, NB, T, R0 + 256>(tmem, da, db0, ks, acc);
    }
}
template <int S, int NB, int KT, int T>
__device__ __forceinline__ void issue_digits(uint32_t tmem, uint64_t da0, uint64_t db0, int ks, uint32_t fresh) {
    if constexpr (T < S) {
        const uint64_t da = da0 + static_cast<uint64_t>((T * KT + ks * 32) >> 4);
        // the first digit writes every accumulator: it starts the chunk's sums on its first K16
        issue_digit<S, NB, T, 0>(tmem, da, db0, ks, (T == 0 && ks == 0) ? fresh : 1u);
        issue_digits<S, NB, KT, T + 1>(tmem, da0, db0, ks, fresh);
    }
}

template <int S, int NC>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_split(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmArgs p) {
    constexpr bool EXACT = split_exact_mode<NC>();
    // TMEM accumulators: one per scale (EXACT), else four or five with a tail; BANDS x 2NC <= 512
    constexpr int BANDS = EXACT ? S : (NC == kSplitBNc ? 4 : 5);
    constexpr int NB = 2 * NC;                       // accumulator columns per band (Re | Im)
    constexpr int CW = NC / 4;                       // complex columns per epilogue warp
    constexpr int kTileB = tile_bytes_b<NC>();
    constexpr int kStage = stage_bytes<S, NC>();
    constexpr int STAGES = split_stages<S, NC>();
    constexpr uint32_t kId = idesc_bf16(NB);
    static_assert(BANDS * NB <= 512, "accumulators exceed TMEM");
    static_assert(CW % 2 == 0, "epilogue column groups read TMEM in pairs of columns");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * kStage);
    uint64_t* full = bars;                 // [STAGES]
    uint64_t* empty = bars + kSplitMaxStages;  // [STAGES]
    uint64_t* chunk_full = bars + 2 * kSplitMaxStages;
    uint64_t* tmem_free = chunk_full + 1;
    uint64_t* mma_done = chunk_full + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(chunk_full + 3);
    volatile int* abort = reinterpret_cast<volatile int*>(chunk_full + 4);
    // tile queue: the producer claims tiles and hands them to the MMA thread and the epilogue
    uint64_t* tq_full = chunk_full + 5;    // [kTileQueue] tile written (producer arrives)
    uint64_t* tq_empty = tq_full + kTileQueue;  // [kTileQueue] read by the MMA thread and the epilogue
    volatile int64_t* tq = reinterpret_cast<volatile int64_t*>(tq_empty + kTileQueue);  // [kTileQueue]
    volatile int64_t* epi_w = tq + kTileQueue;  // the epilogue's current tile, broadcast
    static_assert(2 * kSplitMaxStages + 5 + 3 * kTileQueue + 1 <= 32, "barriers overflow their 256 bytes");
    int* sm_ea = reinterpret_cast<int*>(bars + 32);  // [128] exponents of the current tile's rows
    int* sm_eb = sm_ea + 128;                         // [64] exponents of its complex columns

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // Persistent with dynamic tiles: CTA b starts with work item b and then claims the next
    // unstarted item from a counter (work = pole * tcount + tile), so tiles start in list order
    // whatever the durations of the tiles before them.  The tiles that share an operand tile are
    // adjacent in the list, hence start together and read each K-block of it from L2 within a
    // short window; a fixed round-robin assignment drifted apart on launches whose items have
    // different K and re-read shared operand tiles from DRAM.
    const int64_t n_work = p.tcount * p.np;
    int* claim = p.status + 2;  // [0] items claimed beyond the first wave, [1] CTAs finished
    auto tile_of = [&](int64_t w) { return p.tiles[p.tfirst + w % p.tcount]; };
    auto nkb_of = [&](const GemmTile& t) { return 2 * p.sitems[p.ifirst + t.item].Kpad / kSplitKB; };

    if (threadIdx.x == 0) {
#pragma unroll
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        mbar_init(chunk_full, 1);
        mbar_init(tmem_free, kEpiWarps);
        mbar_init(mma_done, 1);
#pragma unroll
        for (int i = 0; i < kTileQueue; ++i) {
            mbar_init(&tq_full[i], 1);
            mbar_init(&tq_empty[i], 2);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_holder, 512);
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    auto a_tile = [&](int stage, int t) { return smem + stage * kStage + t * kTileBytes; };
    auto b_tile = [&](int stage, int u) { return smem + stage * kStage + S * kTileBytes + u * kTileB; };

    if (warp == 0) {
        if (lane == 0) {
            // producer: one ring of STAGES stages across all of this CTA's tiles
            int64_t g = 0;      // K-blocks issued so far (all tiles)
            int64_t armed = 0;
            for (int64_t jt = 0;; ++jt) {
                const int slot = static_cast<int>(jt % kTileQueue);
                if (jt >= kTileQueue &&
                    !mbar_wait(&tq_empty[slot], static_cast<uint32_t>(((jt / kTileQueue) - 1) & 1), abort))
                    break;
                int64_t w = jt == 0 ? static_cast<int64_t>(blockIdx.x) : gridDim.x + static_cast<int64_t>(atomicAdd(claim, 1));
                if (w >= n_work || *abort) w = -1;
                tq[slot] = w;
                mbar_arrive(&tq_full[slot]);
                if (w < 0) break;
                const GemmTile tile = tile_of(w);
                const int64_t pole = w / p.tcount;
                const SplitItem si = p.sitems[p.ifirst + tile.item];
                const int nkb = nkb_of(tile);
                const int yA0 = static_cast<int>(pole * p.rowsA + si.rowA + tile.m0);
                const int yB0 = static_cast<int>(pole * p.rowsB + si.rowB + (tile.n0 / NC) * NB);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int stage = static_cast<int>(g % STAGES);
                    if (g >= STAGES &&
                        !mbar_wait(&empty[stage], static_cast<uint32_t>(((g / STAGES) - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[stage], kStage);
#pragma unroll
                    for (int t = 0; t < S; ++t)
                        tma_load_2d(a_tile(stage, t), &tmA, kb * kSplitKB, yA0 + t * si.Mpad, &full[stage]);
#pragma unroll
                    for (int u = 0; u < S; ++u)
                        tma_load_2d(b_tile(stage, u), &tmB, kb * kSplitKB, yB0 + u * 2 * si.Npad, &full[stage]);
                    armed = g + 1;
                }
                if (!ok) break;
            }
            if (*abort) {
                // drain: wait for the last (up to STAGES) armed stages' copies to land
                for (int64_t k = armed > STAGES ? armed - STAGES : 0; k < armed; ++k)
                    mbar_wait_drain(&full[k % STAGES], static_cast<uint32_t>((k / STAGES) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issue: chunks are numbered across tiles; chunk c > 0 starts once the epilogue
            // has read chunk c - 1 out of TMEM (which may belong to the previous tile)
            int64_t g = 0, c = 0;
            bool ok = true;
            for (int64_t jt = 0; ok; ++jt) {
                const int slot = static_cast<int>(jt % kTileQueue);
                if (!mbar_wait(&tq_full[slot], static_cast<uint32_t>((jt / kTileQueue) & 1), abort)) break;
                const int64_t w = tq[slot];
                mbar_arrive(&tq_empty[slot]);
                if (w < 0) break;
                const int nkb = nkb_of(tile_of(w));
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int stage = static_cast<int>(g % STAGES);
                    if (!mbar_wait(&full[stage], static_cast<uint32_t>((g / STAGES) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const bool first_in_chunk = (kb % kSplitChunkKB) == 0;
                    if (first_in_chunk && c > 0) {
                        if (!mbar_wait(tmem_free, static_cast<uint32_t>((c - 1) & 1), abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    // Descriptors of this stage's slice tiles: the start-address field is the low
                    // 14 bits (address >> 4), so tile t and K16 half ks are compile-time offsets
                    // from the stage's first tile.  The loops unroll completely (S is a template
                    // parameter), leaving one 64-bit add and one tcgen05.mma per instruction.
                    const uint64_t da0 = sdesc_sw(smem_u32(a_tile(stage, 0)));
                    const uint64_t db0 = sdesc_sw(smem_u32(b_tile(stage, 0)));
                    const uint32_t fresh = first_in_chunk ? 0u : 1u;
                    if constexpr (EXACT) {
#pragma unroll
                        for (int ks = 0; ks < kK16Steps; ++ks) issue_digits<S, NB, kTileBytes, 0>(tmem, da0, db0, ks, fresh);
                    } else {
                        // tail band BANDS-1: slice pairs with t+u >= BANDS+1 (1-based), read out per
                        // chunk like the others
#pragma unroll
                        for (int t = 0; t < S; ++t)
#pragma unroll
                            for (int u = 0; u < S; ++u) {
                                if (t + u > S - 1 || t + u < BANDS - 1) continue;
                                const bool lead = (t + u == BANDS - 1) && t == 0;  // first tail product of a K-block
#pragma unroll
                                for (int ks = 0; ks < kK16Steps; ++ks) {
                                    const uint64_t da = da0 + static_cast<uint64_t>((t * kTileBytes + ks * 32) >> 4);
                                    const uint64_t db = db0 + static_cast<uint64_t>((u * kTileB + ks * 32) >> 4);
                                    umma_bf16(tmem + (BANDS - 1) * NB, da, db, kId, (lead && ks == 0) ? fresh : 1u);
                                }
                            }
                        // exact bands 0..BANDS-2: t+u = 2 .. BANDS (1-based), one scale each
#pragma unroll
                        for (int band = 0; band < BANDS - 1; ++band) {
#pragma unroll
                            for (int t = 0; t < S; ++t) {
                                const int u = band - t;
                                if (u < 0 || u >= S) continue;
#pragma unroll
                                for (int ks = 0; ks < kK16Steps; ++ks) {
                                    const uint64_t da = da0 + static_cast<uint64_t>((t * kTileBytes + ks * 32) >> 4);
                                    const uint64_t db = db0 + static_cast<uint64_t>((u * kTileB + ks * 32) >> 4);
                                    umma_bf16(tmem + band * NB, da, db, kId, (t == 0 && ks == 0) ? fresh : 1u);
                                }
                            }
                        }
                    }
                    umma_commit(&empty[stage]);
                    if ((kb % kSplitChunkKB) == kSplitChunkKB - 1 || kb == nkb - 1) {
                        umma_commit(chunk_full);
                        ++c;
                    }
                }
            }
            umma_commit(mma_done);
        }
    } else {
        // epilogue: warp quarter q reads TMEM lanes 32q..32q+31 (tile rows); column group cg the
        // complex columns cg*CW .. cg*CW+CW-1, i.e. accumulator columns cg*CW.. (Re) and NC+cg*CW..
        // (Im), so that every thread holds whole complex elements.  After a tile's last chunk TMEM
        // is released at once and the conversion to FP64 and the store run from registers while
        // the MMAs of the next tile proceed.
        const int q = warp & 3;
        const int cg = (warp - 2) >> 2;
        const int et = threadIdx.x - 64;
        const bool neg_alpha = p.neg_alpha != 0, add_c = p.add_c != 0;
        int64_t c = 0;  // chunks consumed (all tiles)
        for (int64_t jt = 0;; ++jt) {
            // one thread takes the next tile from the queue and broadcasts it, so every epilogue
            // thread leaves the loop at the same tile (no thread waits at a barrier alone)
            if (et == 0) {
                const int slot = static_cast<int>(jt % kTileQueue);
                int64_t wv = -1;
                if (mbar_wait(&tq_full[slot], static_cast<uint32_t>((jt / kTileQueue) & 1), abort)) {
                    wv = tq[slot];
                    mbar_arrive(&tq_empty[slot]);
                }
                *epi_w = wv;
            }
            // also: this tile's scale exponents may now be written (the previous tile's are no
            // longer read)
            asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
            const int64_t w = *epi_w;
            if (w < 0) break;
            const GemmTile tile = tile_of(w);
            const int64_t pole = w / p.tcount;
            const GemmItem it = p.items[p.ifirst + tile.item];
            const SplitItem si = p.sitems[p.ifirst + tile.item];
            const int nchunks = (nkb_of(tile) + kSplitChunkKB - 1) / kSplitChunkKB;
            double2* Cp = p.C + pole * p.sC + it.c_off;
            if (et < 128) {
                const int m = tile.m0 + et;
                sm_ea[et] = m < it.M ? p.expA[pole * p.erowsA + si.erowA + m] : 0;
            } else if (et < 128 + NC) {
                const int n = tile.n0 + et - 128;
                sm_eb[et - 128] = n < it.N ? p.expB[pole * p.erowsB + si.erowB + n] : 0;
            }
            if (add_c) {
                // pull the C block the final update reads towards L2 while the MMAs run
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int line = et + u * kEpiWarps * 32;  // NC columns x 16 lines of 128 B
                    const int j = line >> 4, r = (line & 15) * 8;
                    const int m = tile.m0 + r, n = tile.n0 + j;
                    if (j < NC && m < it.M && n < it.N && !(p.lower && n > tile.m0 + 127))
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(Cp + m + static_cast<int64_t>(n) * it.ldc));
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
            bool ok = true;
            float hi[2 * CW], lo[2 * CW];  // [0, CW): Re, [CW, 2CW): Im of this warp's columns
#pragma unroll
            for (int j = 0; j < 2 * CW; ++j) {
                hi[j] = 0.f;
                lo[j] = 0.f;
            }
            for (int k = 0; k < nchunks; ++k, ++c) {
                if (!mbar_wait(chunk_full, static_cast<uint32_t>(c & 1), abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // A band's Re and Im columns are requested together and awaited once; with two
                // buffers the next band's loads are in flight while this band's sums run.  TMEM goes
                // back to the MMA warp as soon as the last band is in registers.
                auto load_band = [&](int band, uint32_t* r) {
#pragma unroll
                    for (int part = 0; part < 2; ++part)  // Re columns, then the matching Im columns
                        tmem_ld_cols_async<CW>(tmem + (static_cast<uint32_t>(32 * q) << 16) + band * NB +
                                                   part * NC + cg * CW,
                                               r + part * CW);
                };
                auto release = [&]() {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tmem_free);
                };
                auto sum_band = [&](const uint32_t* r) {
#pragma unroll
                    for (int i = 0; i < 2 * CW; ++i) ff_add(hi[i], lo[i], __uint_as_float(r[i]));
                };
                (void)load_band;
                (void)sum_band;
                if constexpr (kEpiDoubleBuffer<CW>) {
                    uint32_t r[2][2 * CW];
                    load_band(0, r[0]);
                    tmem_wait_ld<2 * CW>(r[0]);
#pragma unroll
                    for (int band = 0; band < BANDS; ++band) {
                        if (band + 1 < BANDS) load_band(band + 1, r[(band + 1) & 1]);
                        sum_band(r[band & 1]);
                        if (band + 1 < BANDS) tmem_wait_ld<2 * CW>(r[(band + 1) & 1]);
                        if (band + 1 == BANDS - 1) release();
                    }
                    if constexpr (BANDS == 1) release();
                } else {
                    // wide column groups: one part (Re or Im columns) at a time
#pragma unroll
                    for (int band = 0; band < BANDS; ++band)
#pragma unroll
                        for (int part = 0; part < 2; ++part) {
                            uint32_t r[CW];
                            tmem_ld_cols_async<CW>(tmem + (static_cast<uint32_t>(32 * q) << 16) + band * NB +
                                                       part * NC + cg * CW,
                                                   r);
                            tmem_wait_ld<CW>(r);
                            if (band == BANDS - 1 && part == 1) release();
#pragma unroll
                            for (int i = 0; i < CW; ++i)
                                ff_add(hi[part * CW + i], lo[part * CW + i], __uint_as_float(r[i]));
                        }
                }
            }
            if (epi_any(!ok || *abort)) break;  // the same decision in every epilogue thread
            // C = alpha * 2^e (hi + lo) + beta * C for this thread's row and CW complex columns:
            // alpha is +-1 and beta 0 or 1 (checked at launch), the sign goes onto the integer
            // result and beta = 1 costs the only FP64 instructions.  A warp stores one column's
            // 32 consecutive rows (512 contiguous bytes) per instruction.
            const int r = 32 * q + lane;
            const int m = tile.m0 + r;
            if (m < it.M) {
                const int ea = sm_ea[r] - 14;
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const int jc = cg * CW + j;
                    const int n = tile.n0 + jc;
                    if (n >= it.N || (p.lower && n > m)) continue;
                    double2* dst = Cp + m + static_cast<int64_t>(n) * it.ldc;
                    const int e = ea + sm_eb[jc];
                    double re = ff_to_double_scaled(hi[j], lo[j], e, neg_alpha);
                    double im = ff_to_double_scaled(hi[CW + j], lo[CW + j], e, neg_alpha);
                    if (add_c) {
                        const double2 old = *dst;
                        re += old.x;
                        im += old.y;
                    }
                    *dst = make_double2(re, im);
                }
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        if (*abort) {
            if (lane == 0) mbar_wait_drain(mma_done, 0);
            __syncwarp();
        }
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0) {
        if (*abort) atomicOr(p.status, kStatusTimeout);
        // the last CTA to finish resets the claim counters for the next launch (every CTA has
        // claimed its last item before it gets here)
        __threadfence();
        if (atomicAdd(claim + 1, 1) == static_cast<int>(gridDim.x) - 1) {
            atomicExch(claim, 0);
            atomicExch(claim + 1, 0);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_num_sms = 148;  // multiprocessors of the current device (persistent grid size)

template <int S, int NC>
cudaError_t set_gemm_attr() {
    return cudaFuncSetAttribute(k_gemm_split<S, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                split_smem_bytes<S, NC>());
}
template <int S>
cudaError_t set_attrs() {
    cudaError_t e = set_gemm_attr<S, kSplitBNc>();
    if (e == cudaSuccess) e = set_gemm_attr<S, kSplitBNc5>();
    if (e == cudaSuccess) e = set_gemm_attr<S, kSplitBNcX7>();
    if constexpr (S <= 6)
        if (e == cudaSuccess) e = set_gemm_attr<S, kSplitBNcX>();
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_slice1<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSplitSlice1SmemWide);
}

}  // namespace

cudaError_t split_init() {
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    cudaError_t e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (sms > 0) g_num_sms = sms;
    if ((e = set_attrs<4>()) != cudaSuccess) return e;
    if ((e = set_attrs<5>()) != cudaSuccess) return e;
    if ((e = set_attrs<6>()) != cudaSuccess) return e;
    if ((e = set_attrs<7>()) != cudaSuccess) return e;
    return cudaSuccess;
}

void split_free(SplitBuffers& B) {
    if (B.sliceA) cudaFree(B.sliceA);
    if (B.sliceB) cudaFree(B.sliceB);
    if (B.expA) cudaFree(B.expA);
    if (B.expB) cudaFree(B.expB);
    B = SplitBuffers{};
}

static cudaError_t encode(CUtensorMap* map, void* base, int64_t cols, int64_t rows, int box_rows) {
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(cols * 2)};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(kSplitKB), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          kRowBytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t split_alloc(SplitBuffers& B, const std::vector<SplitStep>& steps, int slices, int np) {
    (void)slices;
    size_t ca = 0, cb = 0, cea = 0, ceb = 0;
    for (const SplitStep& s : steps) {
        ca = std::max(ca, static_cast<size_t>(s.rowsA) * s.Kcols * np);
        cb = std::max(cb, static_cast<size_t>(s.rowsB) * s.Kcols * np);
        cea = std::max(cea, static_cast<size_t>(s.erowsA) * np);
        ceb = std::max(ceb, static_cast<size_t>(s.erowsB) * np);
    }
    if (B.np >= np && B.capA >= ca && B.capB >= cb && !B.tmA.empty()) return cudaSuccess;
    split_free(B);
    cudaError_t e;
    if ((e = cudaMalloc(&B.sliceA, std::max<size_t>(ca, 64) * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&B.sliceB, std::max<size_t>(cb, 64) * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&B.expA, std::max<size_t>(cea, 1) * 4)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&B.expB, std::max<size_t>(ceb, 1) * 4)) != cudaSuccess) return e;
    B.capA = ca;
    B.capB = cb;
    B.capEA = cea;
    B.capEB = ceb;
    B.np = np;
    B.tmA.assign(steps.size(), CUtensorMap{});
    B.tmB.assign(steps.size(), CUtensorMap{});
    for (size_t i = 0; i < steps.size(); ++i) {
        const SplitStep& s = steps[i];
        if ((e = encode(&B.tmA[i], B.sliceA, s.Kcols, std::max<int64_t>(s.rowsA * np, 128), kSplitBM)) != cudaSuccess)
            return e;
        if ((e = encode(&B.tmB[i], B.sliceB, s.Kcols, std::max<int64_t>(s.rowsB * np, 128), 2 * s.nc)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template <int S>
static cudaError_t run_slice(const Launch& l, const GemmItem* items_dev, const SplitItem* sitems_dev,
                             const SliceBlock* blocks_dev, const SplitStep& step, const SplitBuffers& B,
                             const double2* Abuf, int64_t sA, const double2* Bbuf, int64_t sB, int np,
                             cudaStream_t st) {
    SliceArgs sa{items_dev, sitems_dev, blocks_dev, step.sa_first, l.first, Abuf, sA, l.opA, 0,
                 B.sliceA, step.rowsA, step.Kcols, B.expA, step.erowsA, step.slice_rows, step.slice_ldt, step.nc};
    SliceArgs sb{items_dev, sitems_dev, blocks_dev, step.sb_first, l.first, Bbuf, sB, l.opB, 1,
                 B.sliceB, step.rowsB, step.Kcols, B.expB, step.erowsB, step.slice_rows, step.slice_ldt, step.nc};
    if (step.slice_ldt > 0) {
        const size_t sm = static_cast<size_t>(step.slice_rows) * step.slice_ldt * sizeof(double2);
        k_slice1<S><<<dim3(static_cast<unsigned>(step.sa_count), np), 256, sm, st>>>(sa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_slice1<S><<<dim3(static_cast<unsigned>(step.sb_count), np), 256, sm, st>>>(sb);
        return cudaGetLastError();
    }
    k_slice<S><<<dim3(static_cast<unsigned>(step.sa_count), np), 256, 0, st>>>(sa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_slice<S><<<dim3(static_cast<unsigned>(step.sb_count), np), 256, 0, st>>>(sb);
    return cudaGetLastError();
}

template <int S>
static cudaError_t run_mma(const Launch& l, int step_index, const GemmItem* items_dev,
                           const SplitItem* sitems_dev, const GemmTile* stiles_dev, const SplitStep& step,
                           const SplitBuffers& B, double2* Cbuf, int64_t sC, int np, int* status,
                           cudaStream_t st) {
    if ((l.alpha != 1.0 && l.alpha != -1.0) || (l.beta != 0.0 && l.beta != 1.0)) return cudaErrorInvalidValue;
    const GemmArgs ga{items_dev, sitems_dev, stiles_dev, step.tfirst, l.first, step.rowsA, step.rowsB,
                      step.erowsA, step.erowsB, B.expA, B.expB, Cbuf, sC, l.alpha < 0 ? 1 : 0, l.beta != 0.0 ? 1 : 0,
                      l.lower, status, step.tcount, np};
    const int64_t work = step.tcount * np;
    const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(work, g_num_sms)));
    auto go = [&](auto nc_const) {
        constexpr int NC = decltype(nc_const)::value;
        k_gemm_split<S, NC><<<grid, kThreads, split_smem_bytes<S, NC>(), st>>>(B.tmA[step_index], B.tmB[step_index], ga);
        return cudaGetLastError();
    };
    switch (step.nc) {
        case kSplitBNc: return go(std::integral_constant<int, kSplitBNc>{});
        case kSplitBNc5: return go(std::integral_constant<int, kSplitBNc5>{});
        case kSplitBNcX7: return go(std::integral_constant<int, kSplitBNcX7>{});
        case kSplitBNcX:
            if constexpr (S <= 6) return go(std::integral_constant<int, kSplitBNcX>{});
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t split_slice_step(const Launch& l, const GemmItem* items_dev, const SplitItem* sitems_dev,
                             const SliceBlock* blocks_dev, const SplitStep& step, const SplitBuffers& B,
                             int slices, const double2* Abuf, int64_t sA, const double2* Bbuf, int64_t sB,
                             int np, cudaStream_t st) {
    switch (slices) {
        case 4: return run_slice<4>(l, items_dev, sitems_dev, blocks_dev, step, B, Abuf, sA, Bbuf, sB, np, st);
        case 5: return run_slice<5>(l, items_dev, sitems_dev, blocks_dev, step, B, Abuf, sA, Bbuf, sB, np, st);
        case 6: return run_slice<6>(l, items_dev, sitems_dev, blocks_dev, step, B, Abuf, sA, Bbuf, sB, np, st);
        case 7: return run_slice<7>(l, items_dev, sitems_dev, blocks_dev, step, B, Abuf, sA, Bbuf, sB, np, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t split_mma_step(const Launch& l, int step_index, const GemmItem* items_dev,
                           const SplitItem* sitems_dev, const GemmTile* stiles_dev, const SplitStep& step,
                           const SplitBuffers& B, int slices, double2* Cbuf, int64_t sC, int np, int* status,
                           cudaStream_t st) {
    switch (slices) {
        case 4: return run_mma<4>(l, step_index, items_dev, sitems_dev, stiles_dev, step, B, Cbuf, sC, np, status, st);
        case 5: return run_mma<5>(l, step_index, items_dev, sitems_dev, stiles_dev, step, B, Cbuf, sC, np, status, st);
        case 6: return run_mma<6>(l, step_index, items_dev, sitems_dev, stiles_dev, step, B, Cbuf, sC, np, status, st);
        case 7: return run_mma<7>(l, step_index, items_dev, sitems_dev, stiles_dev, step, B, Cbuf, sC, np, status, st);
        default: return cudaErrorInvalidValue;
    }
}

double split_executed_flops(const Plan& P, const SplitStep& step, const std::vector<SplitItem>& items,
                            const std::vector<GemmTile>& tiles, const Launch& l, int slices) {
    // real MACs issued by the tensor cores: per tile 128 x 2nc x (2 Kpad) per slice pair
    const int pairs = slices * (slices + 1) / 2;
    double macs = 0;
    for (int64_t t = step.tfirst; t < step.tfirst + step.tcount; ++t) {
        const SplitItem& si = items[l.first + tiles[t].item];
        macs += 128.0 * (2.0 * step.nc) * 2.0 * si.Kpad * pairs;
    }
    (void)P;
    return 2.0 * macs;
}

}  // namespace ndsi
