// Tensor-core products on sm_103a (tcgen05): D = A B with FP32 operands, near FP32 accuracy
// by the 3xTF32 split (hi = x rounded to the nearest TF32, lo = x - hi rounded to the nearest
// TF32, so |x - hi - lo| <= 2^-22 |x|; the product is hi_a hi_b + hi_a lo_b + lo_a hi_b, the
// dropped lo_a lo_b term is at most 2^-22 |a b|), accumulated in FP32 in tensor memory.
//
// The whole CTA (NT threads) runs a product: it stages 128-row tiles of A and N-column
// tiles of B, both split, into shared memory in the no-swizzle K-major layout of 8 x 16-byte
// core matrices; thread 0 issues tcgen05.mma (M = 128, N <= 256, K = 8 per instruction)
// with the accumulator in tensor memory and commits to an mbarrier; every warp then reads
// its lane quarter of the accumulator with tcgen05.ld and hands each element to the
// caller's epilogue.  Two stage buffers alternate, so staging chunk i+1 overlaps the
// products of chunk i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tilt {

constexpr int TC_M = 128;          // rows of one accumulator tile (tensor-memory lanes)
constexpr int TC_NMAX = 256;       // columns of the accumulator (tensor-memory columns)
constexpr long long TC_WAIT_LIMIT = 1ll << 22;   // polls of an mbarrier before giving up

// Per-CTA state of the tensor-core path and of the bulk copies (in shared memory).
struct TcState {
    uint64_t mbar[2];      // one mbarrier per stage buffer
    uint64_t jbar;         // completion of the bulk copies of the staged Jacobi sweeps
    uint32_t phase[2];     // parity each mbarrier waits for next
    uint32_t jphase;
    uint32_t tmem;         // tensor-memory base address of the accumulator
    int error;             // non-zero once a bounded wait gave up
};

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- tensor-memory allocation (one full warp executes each of these)
__device__ inline void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the tensor core (async proxy)
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait until the mbarrier completes the phase with the given parity; gives up after
// TC_WAIT_LIMIT polls and returns false.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// ---- bulk copies (the TMA engine's one-dimensional copies), issued by one thread.  Both
// addresses 16-byte aligned, sizes multiples of 16 bytes.
// Arrive on the mbarrier and make its current phase also wait for `bytes` of transfers.
__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared; completion is counted on the mbarrier
__device__ inline void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst_smem)),
                 "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// shared -> global, in the issuing thread's current bulk group
__device__ inline void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem), "r"(smem_u32(src_smem)),
                 "r"(bytes)
                 : "memory");
}
__device__ inline void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread's bulk groups, all but the `n` most recent, have finished reading shared memory
template <int N>
__device__ inline void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
// the issuing thread's bulk groups have completed (their writes are performed)
__device__ inline void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's generic-proxy memory accesses before later async-proxy (bulk copy,
// tensor core) accesses, and async-proxy writes already waited for before later generic ones
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte offset
// (between core matrices adjacent along K), stride-dimension byte offset (between 8-row
// groups), descriptor version 1, no swizzle.
__device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major,
// M x N tile.
__host__ __device__ inline uint32_t idesc_tf32(int M, int N) {
    uint32_t d = 0;
    d |= 1u << 4;                        // D format: F32
    d |= 2u << 7;                        // A format: TF32
    d |= 2u << 10;                       // B format: TF32
    d |= (uint32_t)(N >> 3) << 17;
    d |= (uint32_t)(M >> 4) << 24;
    return d;
}

__device__ inline void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ inline void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns of tensor memory -> 16 registers per thread.
// The load and its wait are one asm statement, so no use of the registers can be scheduled
// before the data has arrived.
__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x rounded to the nearest TF32 value (10 mantissa bits), in an FP32 container.
__device__ inline float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// 3xTF32 split of x: both parts rounded to the nearest TF32 (the tensor core would otherwise
// drop the low 13 mantissa bits of each).
__device__ inline void split_tf32(float x, float& hi, float& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - hi);
}

// Byte offset of element (row r, k) in a no-swizzle K-major tile of `rows` rows: core
// matrix (r / 8, k / 4) at ((k / 4) * rows / 8 + r / 8) * 128, row r % 8 at 16 bytes,
// element k % 4 at 4 bytes.
__device__ inline uint32_t kmajor_off(int r, int k, int rows) {
    return (uint32_t)((((k >> 2) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 3) << 2));
}

// Shared-memory bytes of nbuf stage buffers (each: hi and lo of a 128 x kc tile of A and of
// an Np x kc tile of B) for products of up to Np <= TC_NMAX columns with K chunks of kc.
__host__ __device__ inline size_t tc_stage_bytes(int Np, int kc, int nbuf) {
    return (size_t)nbuf * 2 * (TC_M + Np) * kc * sizeof(float);
}

// Tensor-memory columns for an accumulator of N columns (a power of two >= 32).
__host__ __device__ inline uint32_t tc_tmem_cols(int N) {
    uint32_t c = 32;
    while ((int)c < N) c <<= 1;
    return c;
}

// Set up the tensor-core state: warp 0 allocates ncols columns of tensor memory, thread 0
// initialises the two mbarriers.  All threads.
__device__ inline void tc_setup(TcState* st, uint32_t ncols) {
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&st->tmem, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&st->mbar[0], 1);
        mbar_init(&st->mbar[1], 1);
        mbar_init(&st->jbar, 1);
        st->phase[0] = st->phase[1] = 0;
        st->jphase = 0;
        st->error = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Release the tensor memory (warp 0).  All threads; no product may be in flight.
__device__ inline void tc_teardown(TcState* st, uint32_t ncols) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(st->tmem, ncols);
}

// D (M x N) = A (M x K) B (K x N).  la(m, k) and lb(k, n) return the operand elements (they
// are called only inside the bounds); epi(m, n, value) receives every element of D, exactly
// once, from the thread that read it.  The product runs in tiles of 128 rows x up to
// TC_NMAX columns.  stage: tc_stage_bytes(min(Np, TC_NMAX), kc, nbuf) bytes of shared memory
// (16-byte aligned), Np = N rounded up to 16, kc a multiple of 8, nbuf 1 or 2 (with two
// buffers, staging chunk i+1 overlaps the products of chunk i); the accumulator needs
// tc_tmem_cols(min(Np, TC_NMAX)) columns of tensor memory.  All NTH threads call it.
// Returns false (and sets st->error) when a bounded wait gave up.
// Stage one operand tile (rows x kc, zero outside rows_valid x k_valid) as hi and lo
// K-major core matrices.  Each thread takes four consecutive K elements of one row and
// writes them as one 16-byte row of a core matrix (float4 stores: no bank conflicts).
// KCONTIG: the source is contiguous along K, so consecutive threads take the K quads of one
// row; otherwise consecutive threads take consecutive rows (contiguous in the source).
template <int NTH, bool KCONTIG, class LD>
__device__ __forceinline__ void tc_stage_tile(LD ld, int row0, int rows_valid, int k0, int k_valid, int rows, int kc,
                                              unsigned char* hi, unsigned char* lo) {
    const int nq = kc >> 2;
    for (int idx = threadIdx.x; idx < rows * nq; idx += NTH) {
        int r, kq;
        if (KCONTIG) { kq = idx % nq; r = idx / nq; }
        else { r = idx % rows; kq = idx / rows; }
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = 4 * kq + j;
            x[j] = (r < rows_valid && k0 + k < k_valid) ? ld(row0 + r, k0 + k) : 0.f;
        }
        float h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split_tf32(x[j], h[j], l[j]);
        const uint32_t o = kmajor_off(r, 4 * kq, rows);
        *reinterpret_cast<float4*>(hi + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(lo + o) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

template <int NTH, bool A_KCONTIG, bool B_KCONTIG, class LA, class LB, class EPI>
__device__ __forceinline__ bool tc_gemm(int M, int N, int K, LA la, LB lb, EPI epi, unsigned char* stage, int kc,
                                        int nbuf, TcState* st) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunk = (K + kc - 1) / kc;
    bool ok = __syncthreads_and(st->error == 0);
    for (int n0 = 0; n0 < N && ok; n0 += TC_NMAX) {
        const int Nt = min(N - n0, TC_NMAX);
        const int Np = (Nt + 15) & ~15;
        const size_t abytes = (size_t)TC_M * kc * 4, bbytes = (size_t)Np * kc * 4;
        const uint32_t idesc = idesc_tf32(TC_M, Np);
        for (int m0 = 0; m0 < M && ok; m0 += TC_M) {
            for (int ch = 0; ch < nchunk; ++ch) {
                const int b = nbuf == 2 ? (ch & 1) : 0;
                if (ch >= nbuf && ok) {   // the products of chunk ch - nbuf read this buffer
                    bool w = mbar_wait(&st->mbar[b], st->phase[b]);
                    ok = __syncthreads_and(w && ok);
                    if (threadIdx.x == 0) st->phase[b] ^= 1;
                }
                unsigned char* ahi = stage + (size_t)b * 2 * (abytes + bbytes);
                unsigned char* alo = ahi + abytes;
                unsigned char* bhi = alo + abytes;
                unsigned char* blo = bhi + bbytes;
                const int k0 = ch * kc;
                tc_stage_tile<NTH, A_KCONTIG>(la, m0, M - m0, k0, K, TC_M, kc, ahi, alo);
                auto lbt = [&](int n, int k) { return lb(k, n); };      // B tile stored as N x K
                tc_stage_tile<NTH, B_KCONTIG>(lbt, n0, Nt, k0, K, Np, kc, bhi, blo);
                fence_async_smem();
                __syncthreads();
                if (threadIdx.x == 0 && ok) {
                    tc_fence_after();
                    const uint32_t lbo_a = (uint32_t)(TC_M / 8) * 128, lbo_b = (uint32_t)(Np / 8) * 128;
                    for (int ks = 0; ks < kc / 8; ++ks) {
                        const uint32_t oa = (uint32_t)ks * 2 * lbo_a, ob = (uint32_t)ks * 2 * lbo_b;
                        const uint64_t dah = smem_desc(smem_u32(ahi) + oa, lbo_a, 128);
                        const uint64_t dal = smem_desc(smem_u32(alo) + oa, lbo_a, 128);
                        const uint64_t dbh = smem_desc(smem_u32(bhi) + ob, lbo_b, 128);
                        const uint64_t dbl = smem_desc(smem_u32(blo) + ob, lbo_b, 128);
                        mma_tf32(st->tmem, dah, dbh, idesc, (ch > 0 || ks > 0) ? 1 : 0);
                        mma_tf32(st->tmem, dah, dbl, idesc, 1);
                        mma_tf32(st->tmem, dal, dbh, idesc, 1);
                    }
                    mma_commit(&st->mbar[b]);
                }
            }
            // wait for the products of the last nbuf chunks
            for (int ch = (nchunk >= nbuf ? nchunk - nbuf : 0); ch < nchunk && ok; ++ch) {
                const int b = nbuf == 2 ? (ch & 1) : 0;
                bool w = mbar_wait(&st->mbar[b], st->phase[b]);
                ok = __syncthreads_and(w && ok);
                if (threadIdx.x == 0) st->phase[b] ^= 1;
            }
            __syncthreads();
            tc_fence_after();
            if (!ok) break;
            // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows of the tile)
            // and the 16-column groups wg, wg + NTH/128, ... (wg = w / 4)
            const int q = warp & 3, wg = warp >> 2, ngroups = NTH / 128;
            const int row = m0 + 32 * q + lane;
            for (int c0 = 16 * wg; c0 < Np; c0 += 16 * ngroups) {
                float v[16];
                tmem_ld16(st->tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < Nt) epi(row, n0 + c0 + j, v[j]);
                }
            }
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
    }
    if (!ok && threadIdx.x == 0) st->error = 1;
    __syncthreads();
    return ok;
}

}  // namespace tilt
