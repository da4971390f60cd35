// kgs_conv_tc.cu -- 3x3x3 convolution as an implicit GEMM on the fifth-
// generation tensor cores (tcgen05.mma, accumulator in tensor memory).
//
// GEMM view: out[v][co] = sum over taps t and input channels ci of
// in[v + off(t)][ci] W[t][co][ci].  A CTA owns an 8 (x) by 16 (y) patch of two
// consecutive z-planes: two accumulators of M = 128 rows (voxels) each, all
// output channels (N = cout_p <= 112), so every weight tile that reaches
// shared memory feeds the MMAs of both planes.  The input planes z0 - 1 ..
// z0 + 2 (10 x 18 voxels, all channels each) go through a ring of three
// slots in the K-major no-swizzle layout the MMA reads: 16-byte rows (8
// channels of one voxel), x fastest within a channel octet, so that for every
// tap the 8 x positions of an output row segment are 8 consecutive 16-byte
// rows (one 8 x 16 B core matrix) and the 16 y rows and the channel octets
// are fixed strides.  Each tap is then C/16 MMAs of 128 x N x 16 per plane
// reading shifted windows of the staged planes; no im2col copy is made.  The
// planes move with cp.async: the first two before the pipeline starts, the
// third and fourth by two loader warps while the tensor core works (the
// fourth reuses the first's slot once the taps kz = 0 are done).  The
// weights, packed beforehand so that a tap is one contiguous block in the
// layout the MMA reads, move with one bulk copy per tap into a ring of four
// buffers.  Two threads drive the pipeline without CTA-wide barriers: a
// producer issues the copy of tap t once the MMAs of tap t-4 have released
// its buffer (commit barrier), and an issuer starts the MMAs of tap t once
// its copy has landed (transaction barrier); the remaining threads wait at a
// CTA barrier, not polling, until the issuer has seen the last MMA complete.
// The epilogue reads the accumulators with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = output rows) and applies bias + ReLU, bias only, or the ReLU
// mask of the backward pass.
//
// The weight gradient (wgrad_tc_kernel) is the per-tap GEMM dW[t][co][ci] =
// sum over voxels v of dy[v][co] in[v + off(t)][ci], with the output
// channels in the 128 accumulator lanes (rows past Cout are ignored), the
// input channels as N and the voxels as the reduction dimension.  Both
// stored tensors keep the channels of a voxel contiguous, which for this GEMM
// is the MN-major operand layout (a core matrix is 8 voxels along K by 8
// channels in 16 bytes; instruction-descriptor bits 15 and 16), so tiles move
// with 16-byte cp.async and need no transpose.  A CTA takes the three taps
// that share (kz, ky): three accumulators in tensor memory, and per 8 x 16
// voxel tile one staged dy tile plus one 16 x 10 voxel block of input plane
// z + kz - 1 whose x windows at offsets 0, 1, 2 are the three B operands.
// Three tile buffers rotate (the copies of tile i + 2 in flight while the
// MMAs of tile i run), each released by its commit barrier.  A CTA covers a
// chunk of tiles of one sample and writes its partial; the caller sums the
// partials in a fixed order.
//
// Every wait on a barrier is bounded; on expiry the CTA records the error,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>

#include "kgs_nn.h"

namespace kgs {
namespace nn {
namespace {

constexpr int TX = 8, TY = 16;                 // output patch: 128 voxels = 128 GEMM rows
constexpr int HX = TX + 2, HY = TY + 2, HZ = 3;  // input plane of the patch; ring of HZ plane slots
constexpr int THREADS = 128;
constexpr int OZ = 2;                          // output planes per CTA (two accumulators)
constexpr int TMEM_HALF = 128;                 // columns of one accumulator (>= N)
constexpr int TMEM_COLS = OZ * TMEM_HALF;      // a power of two
constexpr int LOADERS = 64;                    // threads that stream the later input planes
constexpr int NBUF = 4;                        // weight buffers: up to four taps in flight
constexpr long long WAIT_POLLS = 1ll << 20;    // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand without swizzling.
// lbo: bytes between core matrices adjacent along K; sbo: bytes between core
// matrices adjacent along M (or N).  Bits 46-47 hold the descriptor version
// (1 on this architecture family); base offset, LBO mode and layout type 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16
// A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long i = 0; i < WAIT_POLLS; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16-byte asynchronous global -> shared copy; zero-fills when !valid (no
// global read is made then; src must still be a valid address).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory; completion is counted on barrier `bar`.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Weights W[t][co][ci] -> packed[t][ci/8][co][8]: each tap becomes one
// contiguous block in exactly the shared-memory layout the MMA reads, so it
// moves with a single bulk copy.
__global__ void pack_w_kernel(const uint4 *__restrict__ w, int cout_p, int c8n, uint4 *__restrict__ wpk)
{
    const size_t per = (size_t)cout_p * c8n;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 27 * per) return;
    const size_t t = i / per, r = i % per;
    const int co = (int)(r / c8n), c8 = (int)(r % c8n);
    wpk[t * per + (size_t)c8 * cout_p + co] = w[i];
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    conv_tc_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ wpk,
                   const float *__restrict__ bias, void *out, const __nv_bfloat16 *__restrict__ gate, ConvDims dm,
                   int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t full_bar[NBUF], empty_bar[NBUF], done_bar, plane_full[2], plane_empty;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_last;  // a wait gave up; last tap whose MMAs were committed

    const int C8 = dm.cin_p / 8, cout_p = dm.cout_p;
    const uint32_t plane_bytes = (uint32_t)HY * C8 * HX * 16;
    const uint32_t w_bytes = (uint32_t)C8 * cout_p * 16;
    unsigned char *wbuf = sm + HZ * plane_bytes;
    const int tiles_x = (dm.W + TX - 1) / TX;
    const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
    const int z0 = blockIdx.y * OZ, b = blockIdx.z;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    auto full = [&](int t) { return smem_u32(&full_bar[t % NBUF]); };    // weights of tap t landed
    auto empty = [&](int t) { return smem_u32(&empty_bar[t % NBUF]); };  // MMAs of tap t done
    auto use = [](int t) { return (uint32_t)((t / NBUF) & 1); };         // phase parity of tap t's use
    const uint32_t halo_a = smem_u32(sm), w_a = smem_u32(wbuf);
    volatile int *fail = &s_fail;  // written by the pipeline threads
    auto issue_w = [&](int t) {  // bulk copy of tap t into buffer t % NBUF
        mbar_expect_tx(full(t), w_bytes);
        bulk_copy(w_a + (uint32_t)(t % NBUF) * w_bytes, wpk + (size_t)t * cout_p * dm.cin_p, w_bytes, full(t));
    };
    // input plane p (z = z0 - 1 + p, p = 0..3) in slot p % 3: element (hx, hy,
    // channel octet c8) at ((hy * C8 + c8) * HX + hx) * 16
    const size_t vol = (size_t)dm.D * dm.H * dm.W;
    auto load_plane = [&](int p, int first, int stride) {
        const int gz = z0 - 1 + p;
        const uint32_t dst = halo_a + (uint32_t)(p % HZ) * plane_bytes;
        for (int i = first; i < HY * HX * C8; i += stride) {
            const int c8 = i % C8, r = i / C8;
            const int hx = r % HX, hy = r / HX;
            const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
            const bool valid = gx >= 0 && gy >= 0 && gz >= 0 && gx < dm.W && gy < dm.H && gz < dm.D;
            const __nv_bfloat16 *src =
                valid ? in + ((size_t)b * vol + ((size_t)gz * dm.H + gy) * dm.W + gx) * dm.cin_p + c8 * 8 : in;
            cp_async16(dst + (uint32_t)((hy * C8 + c8) * HX + hx) * 16, src, valid);
        }
        cp_async_commit();
    };

    if (threadIdx.x == 0) {
        for (int q = 0; q < NBUF; q++) {
            mbar_init(smem_u32(&full_bar[q]), 1);
            mbar_init(smem_u32(&empty_bar[q]), 1);
        }
        mbar_init(smem_u32(&done_bar), 1);
        mbar_init(smem_u32(&plane_full[0]), LOADERS);
        mbar_init(smem_u32(&plane_full[1]), LOADERS);
        mbar_init(smem_u32(&plane_empty), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_last = -1;
        // the first NBUF taps need no free buffer: start them now
        for (int t = 0; t < NBUF; t++) issue_w(t);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the first two input planes, by every thread
    load_plane(0, threadIdx.x, THREADS);
    load_plane(1, threadIdx.x, THREADS);
    cp_async_wait<0>();
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    int issued = NBUF - 1;  // last tap whose weight copy was issued (thread 0)
    if (threadIdx.x == 0) {
        // producer: tap t reuses the buffer of tap t - NBUF once its MMAs are done
        for (int t = NBUF; t < 27; t++) {
            if (*fail || !mbar_wait(empty(t - NBUF), use(t - NBUF))) {
                *fail = 1;
                break;
            }
            issue_w(t);
            issued = t;
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer: per tap and channel pair, one MMA of 128 x N x 16 for
        // each output plane, both reading the same weights
        const uint32_t tmem = tmem_base;
        const uint32_t idesc = instr_desc(128, cout_p);
        const uint32_t a_lbo = HX * 16, a_sbo = (uint32_t)C8 * HX * 16;
        const uint32_t b_lbo = (uint32_t)cout_p * 16, b_sbo = 8 * 16;
        for (int t = 0; t < 27; t++) {
            const int kx = t % 3, ky = (t / 3) % 3, kz = t / 9;
            // plane kz + 1 (for the second output plane) first used by the taps kz
            bool ok = !*fail;
            if (ok && t == 9) ok = mbar_wait(smem_u32(&plane_full[0]), 0);
            if (ok && t == 18) ok = mbar_wait(smem_u32(&plane_full[1]), 0);
            if (!ok || !mbar_wait(full(t), use(t))) {
                *fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t pa0 = halo_a + (uint32_t)(kz % HZ) * plane_bytes;        // plane kz: output z0
            const uint32_t pa1 = halo_a + (uint32_t)((kz + 1) % HZ) * plane_bytes;  // plane kz + 1: output z0 + 1
            for (int kc = 0; kc < C8 / 2; kc++) {
                const uint32_t off = (uint32_t)(((ky * C8 + 2 * kc) * HX + kx) * 16);
                const uint64_t bd =
                    smem_desc(w_a + (uint32_t)(t % NBUF) * w_bytes + (uint32_t)(2 * kc * cout_p * 16), b_lbo, b_sbo);
                tc_mma(tmem, smem_desc(pa0 + off, a_lbo, a_sbo), bd, idesc, (t | kc) != 0);
                tc_mma(tmem + TMEM_HALF, smem_desc(pa1 + off, a_lbo, a_sbo), bd, idesc, (t | kc) != 0);
            }
            tc_commit(empty(t));
            if (t == 8) tc_commit(smem_u32(&plane_empty));  // plane 0 (slot 0) no longer read
            s_last = t;
        }
        tc_commit(smem_u32(&done_bar));  // all MMAs issued by this thread
        // all MMAs of the CTA are complete once the done barrier has fired.
        // Only this thread waits for it; the others are parked at the CTA
        // barrier below instead of polling beside the pipeline threads.
        if (!mbar_wait(smem_u32(&done_bar), 0)) *fail = 1;
    } else if (threadIdx.x >= THREADS - LOADERS) {
        // loaders: plane 2 into slot 2 now, plane 3 into slot 0 once the MMAs
        // of the taps kz = 0 have released plane 0
        const int lt = threadIdx.x - (THREADS - LOADERS);
        load_plane(2, lt, LOADERS);
        cp_async_wait<0>();
        fence_async_smem();
        mbar_arrive(smem_u32(&plane_full[0]));
        if (mbar_wait(smem_u32(&plane_empty), 0)) {
            load_plane(3, lt, LOADERS);
            cp_async_wait<0>();
            fence_async_smem();
        } else {
            *fail = 1;  // the issuer's wait on plane_full[1] then gives up too
        }
        mbar_arrive(smem_u32(&plane_full[1]));
    }
    __syncthreads();  // the outcome in s_fail / s_last is uniform after it
    const int last = s_last;
    const uint32_t tmem = tmem_base;
    tc_fence_after();
    if (s_fail || last != 26) {
        if (threadIdx.x == 0) {
            atomicExch(err, 1);
            // weight copies issued but never consumed land before the CTA
            // leaves (bounded; at most NBUF are outstanding, on distinct barriers)
            for (int t = last + 1; t <= issued; t++) (void)mbar_wait(full(t), use(t));
        }
    } else {
        const int row = warp * 32 + lane;
        const int vx = x0 + row % TX, vy = y0 + row / TX;
        const bool inside = vx < dm.W && vy < dm.H;
        for (int oz = 0; oz < OZ; oz++) {
            const int z = z0 + oz;
            if (z >= dm.D) break;  // uniform over the CTA
            const size_t vo = (size_t)b * vol + ((size_t)z * dm.H + vy) * dm.W + vx;
            for (int c0 = 0; c0 < cout_p; c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(oz * TMEM_HALF + c0), v);  // all lanes
                if (!inside) continue;
                if (MODE == 1) {
                    float *o = static_cast<float *>(out) + vo * cout_p + c0;
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4 *>(o + i) =
                            make_float4(v[i] + bias[c0 + i], v[i + 1] + bias[c0 + i + 1], v[i + 2] + bias[c0 + i + 2],
                                        v[i + 3] + bias[c0 + i + 3]);
                } else {
                    __align__(16) __nv_bfloat162 h[8];
                    if (MODE == 0) {
#pragma unroll
                        for (int i = 0; i < 8; i++)
                            h[i] = __floats2bfloat162_rn(fmaxf(v[2 * i] + bias[c0 + 2 * i], 0.f),
                                                         fmaxf(v[2 * i + 1] + bias[c0 + 2 * i + 1], 0.f));
                    } else {
                        __align__(16) __nv_bfloat162 g[8];
                        const uint4 *gp = reinterpret_cast<const uint4 *>(gate + vo * cout_p + c0);
                        reinterpret_cast<uint4 *>(g)[0] = gp[0];
                        reinterpret_cast<uint4 *>(g)[1] = gp[1];
#pragma unroll
                        for (int i = 0; i < 8; i++)
                            h[i] = __floats2bfloat162_rn(__bfloat162float(g[i].x) > 0.f ? v[2 * i] : 0.f,
                                                         __bfloat162float(g[i].y) > 0.f ? v[2 * i + 1] : 0.f);
                    }
                    uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out) + vo * cout_p + c0);
                    o[0] = reinterpret_cast<uint4 *>(h)[0];
                    o[1] = reinterpret_cast<uint4 *>(h)[1];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient: part[b][chunk][t][co][ci] = sum over the chunk's voxels v
// of dy[v][co] * in[v + off(t)][ci], per tap a tcgen05 GEMM with M = co (128
// TMEM lanes, rows >= cout_p ignored), N = ci and K = voxels in steps of 16.
// Both tensors store the channels of a voxel contiguously, which for this
// GEMM is the MN-major operand layout: a core matrix is 8 voxels (along K) x
// 8 channels (16 bytes), so tiles move with 16-byte asynchronous copies and
// need no transpose.  A CTA takes the three taps that share (kz, ky) -- three
// accumulators in tensor memory -- for a chunk of 8 x 16-voxel tiles.  Per
// tile it stages dy of the tile, [y][co/8][x][16 B], and rows y0 + ky - 1 ..
// y0 + ky + 14, columns x0 - 1 .. x0 + 8 of input plane z + kz - 1,
// [y][ci/8][x][16 B]; the windows of that block at x offsets 0, 1, 2 are the
// B operands of the three taps.  Three tile buffers rotate: the copies of
// tile i + 2 are in flight while the tensor core works on tile i.
constexpr int WG_TILES = 32;  // voxel tiles of 128 per CTA
constexpr int WG_BUF = 3;     // tile buffers
constexpr int WG_TMEM = 512;  // three accumulators of 128 columns

// kind::f16 instruction descriptor with both operands MN-major (bits 15, 16).
__host__ __device__ constexpr uint32_t instr_desc_mn(int M, int N)
{
    return instr_desc(M, N) | (1u << 15) | (1u << 16);
}

struct WgLayout {
    uint32_t a_bytes, h_bytes, buf_bytes, total;
};
// Shared memory of the weight-gradient CTA: WG_BUF x (dy tile, input block),
// then a pad such that every MMA read stays inside the allocation even if
// the two descriptor strides were applied the other way round.
__host__ __device__ inline WgLayout wg_layout(int cin_p, int cout_p)
{
    const int c8o = cout_p / 8, c8i = cin_p / 8;
    WgLayout L;
    L.a_bytes = (uint32_t)(TY * c8o * TX * 16);
    L.h_bytes = (uint32_t)(TY * c8i * HX * 16);
    L.buf_bytes = L.a_bytes + L.h_bytes;
    const int over_a = 13 * c8o * 128 + 256 - (int)L.h_bytes;  // past the buffer end, strides swapped
    const int over_b = c8i * (c8i - 3) * HX * 16 + 2 * HX * 16;
    int pad = 2048;
    if (over_a > pad) pad = over_a;
    if (over_b > pad) pad = over_b;
    L.total = WG_BUF * L.buf_bytes + (uint32_t)pad + 128;
    return L;
}

__global__ void __launch_bounds__(THREADS, 1)
    wgrad_tc_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ dy,
                    float *__restrict__ part, ConvDims dm, int n_chunks, int *err)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar[WG_BUF], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int cout_p = dm.cout_p, cin_p = dm.cin_p, C8o = cout_p / 8, C8i = cin_p / 8;
    const WgLayout L = wg_layout(cin_p, cout_p);
    const uint32_t base = smem_u32(sm);
    const int g = blockIdx.x, chunk = blockIdx.y, b = blockIdx.z;
    const int kz = g / 3, ky = g % 3;  // taps 9 kz + 3 ky + kx, kx = 0, 1, 2
    const int tiles_x = (dm.W + TX - 1) / TX, tiles_y = (dm.H + TY - 1) / TY;
    const int n_tiles = tiles_x * tiles_y * dm.D;
    const int tile0 = chunk * WG_TILES, nt = min(n_tiles, tile0 + WG_TILES) - tile0;
    const size_t vol = (size_t)dm.D * dm.H * dm.W;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (threadIdx.x == 0) {
        for (int q = 0; q < WG_BUF; q++) mbar_init(smem_u32(&bar[q]), 1);
        mbar_init(smem_u32(&done_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(WG_TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc_mn(128, cin_p);

    // asynchronous copies of tile tile0 + i into buffer i % WG_BUF (one group)
    auto load_tile = [&](int i) {
        const int tile = tile0 + i;
        const int tz = tile / (tiles_x * tiles_y), txy = tile % (tiles_x * tiles_y);
        const int x0 = (txy % tiles_x) * TX, y0 = (txy / tiles_x) * TY;
        const uint32_t abuf = base + (uint32_t)(i % WG_BUF) * L.buf_bytes, hbuf = abuf + L.a_bytes;
        for (int k = threadIdx.x; k < TX * TY * C8o; k += THREADS) {
            const int c8 = k % C8o, v = k / C8o, vx = v % TX, vy = v / TX;
            const int gx = x0 + vx, gy = y0 + vy;
            const bool ok = gx < dm.W && gy < dm.H;
            const __nv_bfloat16 *src =
                ok ? dy + ((size_t)b * vol + ((size_t)tz * dm.H + gy) * dm.W + gx) * cout_p + c8 * 8 : dy;
            cp_async16(abuf + (uint32_t)((vy * C8o + c8) * TX + vx) * 16, src, ok);
        }
        const int sz = tz + kz - 1;
        for (int k = threadIdx.x; k < TY * HX * C8i; k += THREADS) {
            const int c8 = k % C8i, h = k / C8i, hx = h % HX, hy = h / HX;
            const int sx = x0 + hx - 1, sy = y0 + hy + ky - 1;
            const bool ok = sz >= 0 && sz < dm.D && sx >= 0 && sx < dm.W && sy >= 0 && sy < dm.H;
            const __nv_bfloat16 *src =
                ok ? in + ((size_t)b * vol + ((size_t)sz * dm.H + sy) * dm.W + sx) * cin_p + c8 * 8 : in;
            cp_async16(hbuf + (uint32_t)((hy * C8i + c8) * HX + hx) * 16, src, ok);
        }
        cp_async_commit();
    };

    // Thread 0 issues the MMAs and makes every wait on their completion; the
    // other threads wait for it at CTA barriers rather than polling beside it
    // in its warp.  s_fail records a wait that gave up (uniform after a barrier).
    if (threadIdx.x == 0) s_fail = 0;
    for (int i = 0; i < WG_BUF - 1 && i < nt; i++) load_tile(i);
    for (int i = 0; i < nt; i++) {
        const int j = i + WG_BUF - 1;
        if (j < nt) {
            // tile j reuses the buffer of tile i - 1: its MMAs must have completed
            if (i >= 1) {
                if (threadIdx.x == 0 && !s_fail && !mbar_wait(smem_u32(&bar[(i - 1) % WG_BUF]), ((i - 1) / WG_BUF) & 1))
                    s_fail = 1;
                __syncthreads();
            }
            load_tile(j);
            cp_async_wait<WG_BUF - 1>();  // tile i has landed
        } else if (i + 1 < nt) {
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0 && !s_fail) {
            const uint32_t abuf = base + (uint32_t)(i % WG_BUF) * L.buf_bytes, hbuf = abuf + L.a_bytes;
#pragma unroll 1
            for (int ks = 0; ks < TY / 2; ks++) {  // K = 16 voxels: tile rows 2ks, 2ks + 1
                const uint64_t a = smem_desc(abuf + (uint32_t)(2 * ks * C8o * TX) * 16, (uint32_t)(C8o * TX * 16), TX * 16);
#pragma unroll
                for (int kx = 0; kx < 3; kx++) {
                    const uint64_t bd =
                        smem_desc(hbuf + (uint32_t)(2 * ks * C8i * HX + kx) * 16, (uint32_t)(C8i * HX * 16), HX * 16);
                    tc_mma(tmem + (uint32_t)(kx * 128), a, bd, idesc, (i | ks) != 0);
                }
            }
            tc_commit(smem_u32(&bar[i % WG_BUF]));
        }
    }
    if (threadIdx.x == 0) {
        tc_commit(smem_u32(&done_bar));
        if (!mbar_wait(smem_u32(&done_bar), 0)) s_fail = 1;
    }
    __syncthreads();
    tc_fence_after();
    if (s_fail) {  // uniform: the loads below are warp-collective
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else {
        // row co = TMEM lane; columns kx * 128 + ci
        const int co = warp * 32 + lane;
        for (int kx = 0; kx < 3; kx++) {
            const int t = (kz * 3 + ky) * 3 + kx;
            float *dst = part + (((size_t)b * n_chunks + chunk) * 27 + t) * cout_p * cin_p;
            for (int c0 = 0; c0 < cin_p; c0 += 16) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kx * 128 + c0), v);
                if (co >= cout_p) continue;
#pragma unroll
                for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4 *>(dst + (size_t)co * cin_p + c0 + k) =
                        make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WG_TMEM) : "memory");
    }
}

template <int MODE>
cudaError_t launch(const __nv_bfloat16 *in, const __nv_bfloat16 *wpk, const float *bias, void *out,
                   const __nv_bfloat16 *gate, ConvDims dm, int *err, cudaStream_t s)
{
    const size_t smem = (size_t)HZ * HY * (dm.cin_p / 8) * HX * 16 + NBUF * (size_t)(dm.cin_p / 8) * dm.cout_p * 16;
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = ((dm.W + TX - 1) / TX) * ((dm.H + TY - 1) / TY);
    conv_tc_kernel<MODE><<<dim3(tiles, (dm.D + OZ - 1) / OZ, dm.B), THREADS, smem, s>>>(in, wpk, bias, out, gate, dm,
                                                                                     err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t conv_tc(int mode, const __nv_bfloat16 *in, const __nv_bfloat16 *w, __nv_bfloat16 *wpk, const float *bias,
                    void *out, const __nv_bfloat16 *gate, ConvDims dm, int *err, cudaStream_t s)
{
    if (dm.cin_p % 16 || dm.cout_p % 16 || dm.cin_p < 16 || dm.cout_p < 16 || dm.cin_p > 112 || dm.cout_p > 112)
        return cudaErrorInvalidValue;
    const size_t n16 = (size_t)27 * dm.cout_p * (dm.cin_p / 8);
    pack_w_kernel<<<(unsigned)((n16 + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4 *>(w), dm.cout_p,
                                                                 dm.cin_p / 8, reinterpret_cast<uint4 *>(wpk));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (mode) {
    case 0: return launch<0>(in, wpk, bias, out, gate, dm, err, s);
    case 1: return launch<1>(in, wpk, bias, out, gate, dm, err, s);
    default: return launch<2>(in, wpk, bias, out, gate, dm, err, s);
    }
}

int wgrad_chunks(const ConvDims &dm)
{
    const int tiles = ((dm.W + TX - 1) / TX) * ((dm.H + TY - 1) / TY) * dm.D;
    return (tiles + WG_TILES - 1) / WG_TILES;
}

cudaError_t wgrad_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *dy, float *part, ConvDims dm, int *err,
                     cudaStream_t s)
{
    if (dm.cin_p % 16 || dm.cout_p % 16 || dm.cin_p < 16 || dm.cout_p < 16 || dm.cin_p > 112 || dm.cout_p > 112)
        return cudaErrorInvalidValue;
    // at least 120 KB: one CTA per SM, so no CTA waits for tensor memory held by another
    const size_t smem = std::max<size_t>(wg_layout(dm.cin_p, dm.cout_p).total, 120 * 1024);
    cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int n_chunks = wgrad_chunks(dm);
    wgrad_tc_kernel<<<dim3(9, n_chunks, dm.B), THREADS, smem, s>>>(in, dy, part, dm, n_chunks, err);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace kgs
