// sky_common.cuh -- device helpers shared by libsky's kernels (sm_103a).
//
// Inline PTX for the Blackwell async-copy machinery (mbarrier + 1-D bulk
// copies through the TMA unit), release/acquire flags for the decoupled
// look-back scan, and a few bit tricks. Every wait here is bounded: after
// kWaitLimit polls it records SKY_DEV_ERR_TIMEOUT in the call's error word and
// gives up, so no kernel of this library can spin forever.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sky {

constexpr int kMaxDim = 16;
constexpr unsigned kFull = 0xffffffffu;

// Device error bits (OR-ed into one uint32 per call).
constexpr uint32_t SKY_DEV_ERR_NONFINITE = 1u;
constexpr uint32_t SKY_DEV_ERR_TIMEOUT = 2u;
constexpr uint32_t SKY_DEV_ERR_CAPACITY = 4u;
constexpr uint32_t SKY_DEV_ERR_LAYOUT = 8u;   // a shared-memory table not at the alignment its addressing needs

// Upper bound on polls of any flag or barrier (each poll may suspend briefly).
constexpr uint32_t kWaitLimit = 1u << 22;

// A smaller poll limit for the pipeline waits (those given an error word),
// set by sky_set_wait_limit for tests of the timeout path; 0 = kWaitLimit.
// The waits that let a CTA's own bulk copies land before it exits (no error
// word) always keep kWaitLimit, so a short limit never leaves a copy in
// flight. Every translation unit holds its own copy of the constant and
// registers a setter for it; the library sets them all.
using WaitLimitSetter = cudaError_t (*)(uint32_t);
void register_wait_limit_setter(WaitLimitSetter f);   // sky_api.cu
static __constant__ uint32_t c_wait_limit;
static cudaError_t set_wait_limit_here(uint32_t v) { return cudaMemcpyToSymbol(c_wait_limit, &v, sizeof(v)); }
struct WaitLimitRegistrar {
    explicit WaitLimitRegistrar(WaitLimitSetter f) { register_wait_limit_setter(f); }
};
static const WaitLimitRegistrar g_wait_limit_registrar(&set_wait_limit_here);

__device__ __forceinline__ uint32_t wait_limit(const uint32_t* err)
{
    const uint32_t l = err ? c_wait_limit : 0u;
    return l ? l : kWaitLimit;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a barrier phase. Returns false (and flags a timeout) when
// the limit runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err)
{
    const uint32_t lim = wait_limit(err);
    for (uint32_t i = 0; i < lim; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    if (err) atomicOr(err, SKY_DEV_ERR_TIMEOUT);
    return false;
}

// 1-D bulk copy global -> shared through the TMA unit, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---- per-thread asynchronous copies global -> shared ------------------------
// Fire-and-forget (the thread does not wait for each load); cp_async_wait_all
// then waits for every copy the thread issued. The 16-byte form needs both
// addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- release / acquire flags ----------------------------------------------
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t* p)
{
    return __ldcg(p);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- decoupled look-back (single-pass prefix over tiles) --------------------
// State word per tile: high 32 bits = flag (0 empty, 1 aggregate, 2 inclusive),
// low 32 bits = value. Tiles are numbered in claim order (an atomic counter),
// so every predecessor of a tile belongs to a CTA that is already running and
// the wait below always ends; it is bounded all the same.
constexpr unsigned long long kFlagAgg = 1ull << 32;
constexpr unsigned long long kFlagInc = 2ull << 32;

// Called by all 32 lanes of ONE warp. Returns the exclusive prefix of `tile`.
__device__ __forceinline__ uint32_t lookback_prefix(unsigned long long* states, uint32_t tile,
                                                    uint32_t aggregate, uint32_t* err)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release_u64(&states[0], kFlagInc | aggregate);
        return 0;
    }
    if (lane == 0) st_release_u64(&states[tile], kFlagAgg | aggregate);
    uint32_t exclusive = 0;
    long long base = (long long)tile - 1;
    uint32_t polls = 0;
    const uint32_t lim = wait_limit(err);
    while (true) {
        long long i = base - lane;
        unsigned long long v = (i >= 0) ? ld_acquire_u64(&states[i]) : (kFlagInc | 0ull);
        while (__any_sync(kFull, (v >> 32) == 0)) {
            if (++polls > lim) {
                if (lane == 0 && err) atomicOr(err, SKY_DEV_ERR_TIMEOUT);
                v = kFlagInc;  // give up: the result is flagged as invalid
                break;
            }
            __nanosleep(32);
            if ((v >> 32) == 0) v = ld_acquire_u64(&states[i]);
        }
        const uint32_t inc_mask = __ballot_sync(kFull, (v >> 32) == 2);
        uint32_t val = (uint32_t)(v & 0xffffffffull);
        if (inc_mask) {
            const int first = __ffs(inc_mask) - 1;
            if (lane > first) val = 0;
            for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
            exclusive += val;
            break;
        }
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
        exclusive += val;
        base -= 32;
    }
    if (lane == 0) st_release_u64(&states[tile], kFlagInc | (unsigned long long)(exclusive + aggregate));
    return exclusive;
}

// ---- value -> column map (Eq. 1 with min/max normalisation) ----------------
// t = (x - off) * s in binary32 round-to-nearest with no contraction, then
// floor and clamp to [0, G-1] (the float -> unsigned conversion saturates:
// negative and NaN give 0). Monotone non-decreasing in x.
__device__ __forceinline__ uint32_t column_of(float x, float off, float s, uint32_t G)
{
    const float t = __fmul_rn(__fsub_rn(x, off), s);
    const uint32_t c = __float2uint_rd(t);
    return c < G - 1u ? c : G - 1u;
}

// Order-preserving float <-> uint32 (for atomic min/max on floats).
__device__ __forceinline__ uint32_t float_to_ordered(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__host__ __device__ constexpr inline int pad4(int d) { return (d + 3) & ~3; }

// ---- cell keys -----------------------------------------------------------
// Key of the cell one step down the diagonal is key - ones_key (valid when
// every column of the key is >= 1).
__device__ __forceinline__ uint32_t ones_key(int log2g, int d)
{
    uint32_t o = 0;
    for (int k = 0; k < d; ++k) o |= 1u << (log2g * k);
    return o;
}

__device__ __forceinline__ bool all_columns_positive(uint32_t key, int log2g, int d)
{
    const uint32_t m = (1u << log2g) - 1u;
    bool ok = true;
    for (int k = 0; k < d; ++k) ok &= ((key >> (log2g * k)) & m) != 0u;
    return ok;
}

// Block-wide exclusive scan of one value per thread (NT threads, NT <= 1024).
template <int NT = 256>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < NT / 32) ? s_warp[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[NT / 32 - 1];
    const uint32_t before = warp ? s_warp[warp - 1] : 0u;
    return before + x - v;
}

// Inclusive OR-scan of the len words p[0], p[stride], ... (after OR-ing
// `init` into the first); the loads of a batch are issued before its stores,
// so a long line is not one load -> store chain.
constexpr int kScanBatch = 8;

__device__ __forceinline__ void or_scan_strided(uint32_t* p, uint32_t len, uint32_t stride, uint32_t init)
{
    uint32_t acc = init;
    for (uint32_t j0 = 0; j0 < len; j0 += kScanBatch) {
        uint32_t v[kScanBatch];
#pragma unroll
        for (int u = 0; u < kScanBatch; ++u) v[u] = (j0 + u < len) ? p[(j0 + u) * stride] : 0u;
#pragma unroll
        for (int u = 0; u < kScanBatch; ++u) {
            acc |= v[u];
            if (j0 + u < len) p[(j0 + u) * stride] = acc;
        }
    }
}

// Inclusive prefix-OR along dimension k of the 2^(log2g*d)-bit grid stored in
// `words` 32-bit words (bit stride of dimension k: 2^(log2g*k)). Threads
// tid = 0 .. nthr-1 of the caller share the work; the caller orders
// successive dimensions (grid launches or __syncthreads). Grids hold at most
// 2^27 bits, so word indices fit in 32 bits; every stride and line length is
// a power of two, so indices are split with shifts and masks.
__device__ __forceinline__ void prefix_or_dim(uint32_t* R, int64_t words, int log2g, int k, int64_t tid,
                                              int64_t nthr)
{
    const int slog = log2g * k;
    const uint32_t G = 1u << log2g;
    const uint32_t nw = (uint32_t)words;
    const uint32_t t0 = (uint32_t)tid, nt = (uint32_t)nthr;
    if (slog >= 5) {
        // whole words: word stride sw = 2^ls, G words per line
        const int ls = slog - 5;
        const uint32_t sw = 1u << ls;
        const uint32_t ncol = nw >> log2g;
        for (uint32_t c = t0; c < ncol; c += nt) {
            const uint32_t lo = c & (sw - 1u), hi = c >> ls;
            or_scan_strided(R + ((hi << log2g) << ls) + lo, G, sw, 0u);
        }
    } else if (slog + log2g <= 5) {
        // every line inside one word: log2(G) doubling steps with masks that
        // keep each shifted bit inside its own line (lane b of each warp
        // votes for bit b; callers run whole, converged warps here)
        const uint32_t lane = threadIdx.x & 31u;
        uint32_t mask[6];
        int nsteps = 0;
        for (uint32_t j = 1; j < G; j <<= 1)
            mask[nsteps++] = __ballot_sync(kFull, ((lane >> slog) & (G - 1u)) >= j);
        for (uint32_t w = t0; w < nw; w += nt) {
            uint32_t x = R[w];
            int st = 0;
            for (uint32_t j = 1; j < G; j <<= 1, ++st) x |= (x << (j << slog)) & mask[st];
            R[w] = x;
        }
    } else {
        // a line spans Lw = 2^(slog + log2g - 5) consecutive words holding
        // e = 32 >> slog of its elements each (2^slog interleaved lines): scan
        // inside each word, then carry the last element group from word to word
        const int lw = slog + log2g - 5;
        const uint32_t Lw = 1u << lw;
        const int e = 32 >> slog;
        const int sbits = 1 << slog;
        const uint32_t rep = __ballot_sync(kFull, ((threadIdx.x & 31u) & (uint32_t)(sbits - 1)) == 0u);
        const uint32_t ngroups = nw >> lw;
        for (uint32_t g = t0; g < ngroups; g += nt) {
            uint32_t* p = R + (g << lw);
            uint32_t carry = 0;
            for (uint32_t t0w = 0; t0w < Lw; t0w += kScanBatch) {
                uint32_t v[kScanBatch];
#pragma unroll
                for (int u = 0; u < kScanBatch; ++u) v[u] = (t0w + u < Lw) ? p[t0w + u] : 0u;
#pragma unroll
                for (int u = 0; u < kScanBatch; ++u) {
                    uint32_t x = v[u];
                    for (int j = 1; j < e; j <<= 1) x |= x << (j << slog);
                    x |= carry;
                    if (t0w + u < Lw) p[t0w + u] = x;
                    const uint32_t top = x >> (32 - sbits);
                    carry = top * rep;
                }
            }
        }
    }
}

// Dimensions 0 .. kin-1 at once, all of them lying inside one word
// (log2g * kin <= 5): the per-dimension prefix-ORs commute, so applying them
// one after the other to each word in registers equals kin passes of
// prefix_or_dim. Whole, converged warps only (the masks are lane votes).
__device__ __forceinline__ void prefix_or_inword(uint32_t* R, int64_t words, int log2g, int kin, int64_t tid,
                                                 int64_t nthr)
{
    if (kin <= 0) return;
    const uint32_t G = 1u << log2g;
    const uint32_t lane = threadIdx.x & 31u;
    int nst = 0;
    for (uint32_t j = 1; j < G; j <<= 1) ++nst;
    // [dimension][doubling step], at most 5 x 5, fully unrolled so that the
    // masks stay in registers
    uint32_t mask[5][5];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int st = 0; st < 5; ++st)
            mask[k][st] = __ballot_sync(kFull, k < kin && st < nst &&
                                                   ((lane >> (log2g * k)) & (G - 1u)) >= (1u << st));
    const uint32_t nw = (uint32_t)words;
    for (uint32_t w = (uint32_t)tid; w < nw; w += (uint32_t)nthr) {
        uint32_t x = R[w];
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int st = 0; st < 5; ++st)
                if (k < kin && st < nst) x |= (x << ((1u << st) << (log2g * k))) & mask[k][st];
        R[w] = x;
    }
}

// dominated[c] = prefix[c - (1,..,1)] when every column of c is >= 1 (Def. 3).



}  // namespace sky
