// Learned initialiser: a 3-D U-Net that guesses the relaxed labels from
// atom-density and CFA-field features, so that the flip sweep starts near
// its end (it always finishes from the guess).  The paper starts from tight
// or loose surfaces (Sec. 3.1, "Initial surfaces"); this network is an
// alternative start, trained on label fields that the plain method relaxes.
//
// Network (channels 32, 64, 128, 128; grid dimensions multiples of 8):
//   e0 = relu(conv3(x))            e1 = relu(conv3(pool(e0)))
//   e2 = relu(conv3(pool(e1)))     e3 = relu(conv3(pool(e2)))
//   d2 = relu(conv3([e2, up(e3)])) d1 = relu(conv3([e1, up(d2)]))
//   d0 = relu(conv3([e0, up(d1)])) z  = conv1(d0)
// with 3x3x3 zero-padded cross-correlations, 2x2x2 mean pooling, nearest
// doubling (read in place: the coarse input of a decoder conv is indexed at
// half the fine coordinates) and channel concatenation (two input tensors).
//
// Storage: activations channels-last (cell-major, channels contiguous) in
// bfloat16; weights bfloat16 [tap][cout][cin] for the forward pass and
// [tap][cin][cout] with flipped taps for the input gradient; FP32 master
// weights, gradients and Adam moments in one flat vector.  The convolutions
// are implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16 in, FP32
// accumulate); the rest are plain elementwise and reduction kernels.
#include <cuda.h>
#include <cuda_bf16.h>

#include "vesis_internal.cuh"

namespace vesis {
namespace unet {

typedef __nv_bfloat16 bf16;

constexpr int kLevels = 4;
constexpr int kCh[kLevels] = {32, 64, 128, 128};
constexpr int kInPad = 32;       // input features padded to 32 channels

// ------------------------------------------------------------ mma helpers
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4],
                                         const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld_s32(const bf16 *p)
{
    return *reinterpret_cast<const unsigned *>(p);
}

// ------------------------------------------------------------ convolution
// Implicit GEMM: M = cells (64 per block), N = output channels (BN per
// block), K = 27 taps x input channels in chunks of 32.  The input is the
// concatenation of A (Ca channels at the output's resolution) and B (Cb
// channels at half of it, read at half the coordinates).
struct ConvArgs {
    int nx, ny, nz;
    long long V;
    const bf16 *A;
    int Ca;
    const bf16 *B;
    int Cb;
    const bf16 *Wt;      // [27][Cout][Cin]
    const float *bias;   // Cout or NULL
    int Cout;
    void *Y;             // bf16 [V][Cout] (relu) or float [V][Cout]
    int k16 = 2;         // halves of each 32-channel stage that hold data (the
                         // input layer's 3 features fill only the first)
    // 1x1 head fused into a 32-channel layer's epilogue (TMA kernel only):
    // hz[v] = hb + sum_c hw[c] y_c of the BF16-rounded outputs y, which are
    // then not stored
    const float *hw = nullptr, *hb = nullptr;
    float *hz = nullptr;
    // only the taps at x offset 0 hold weights (the input layer with its x
    // neighbours folded into channels): the TMA kernel skips the others
    bool x1 = false;
};

constexpr int CM = 64;          // cells per block
constexpr int CK = 32;          // input channels per stage
constexpr int SROW = CK + 8;    // padded smem row (conflict-free fragment loads)

template <int BN, bool RAW>
__global__ void __launch_bounds__(128) k_conv(ConvArgs P)
{
    __shared__ __align__(16) bf16 sA[CM][SROW];
    __shared__ __align__(16) bf16 sB[BN][SROW];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const long long v0 = (long long)blockIdx.x * CM;
    const int co0 = blockIdx.y * BN;
    const int Cin = P.Ca + P.Cb;
    const long long nyz = (long long)P.ny * P.nz;
    const int hy = P.ny >> 1, hz = P.nz >> 1;
    // the cell this thread stages
    const int row = t >> 1, half = t & 1;
    const long long v = v0 + row;
    int ci = 0, cj = 0, ck = 0;
    if (v < P.V) {
        ci = (int)(v / nyz);
        const long long rem = v - (long long)ci * nyz;
        cj = (int)(rem / P.nz);
        ck = (int)(rem - (long long)cj * P.nz);
    }
    float acc[BN / 8][4];
#pragma unroll
    for (int n = 0; n < BN / 8; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;

    for (int tap = 0; tap < 27; ++tap) {
        const int da = tap / 9 - 1, db = (tap / 3) % 3 - 1, dc = tap % 3 - 1;
        const int ii = ci + da, jj = cj + db, kk = ck + dc;
        const bool inside = v < P.V && ii >= 0 && ii < P.nx && jj >= 0 && jj < P.ny &&
                            kk >= 0 && kk < P.nz;
        for (int c0 = 0; c0 < Cin; c0 += CK) {
            uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0;
            if (inside) {
                const bf16 *src;
                if (c0 < P.Ca)
                    src = P.A + ((long long)ii * nyz + (long long)jj * P.nz + kk) * P.Ca + c0;
                else
                    src = P.B + (((long long)(ii >> 1) * hy + (jj >> 1)) * hz + (kk >> 1)) * P.Cb +
                          (c0 - P.Ca);
                const uint4 *s4 = reinterpret_cast<const uint4 *>(src + half * 16);
                x0 = s4[0];
                x1 = s4[1];
            }
            uint4 *d4 = reinterpret_cast<uint4 *>(&sA[row][half * 16]);
            d4[0] = x0;
            d4[1] = x1;
            if (t < 2 * BN) {
                const bf16 *src = P.Wt + ((long long)tap * P.Cout + co0 + row) * Cin + c0 + half * 16;
                const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
                uint4 *e4 = reinterpret_cast<uint4 *>(&sB[row][half * 16]);
                e4[0] = s4[0];
                e4[1] = s4[1];
            }
            __syncthreads();
#pragma unroll
            for (int ks = 0; ks < CK; ks += 16) {
                unsigned a[4];
                const int r0 = w * 16 + g;
                a[0] = ld_s32(&sA[r0][ks + 2 * tq]);
                a[1] = ld_s32(&sA[r0 + 8][ks + 2 * tq]);
                a[2] = ld_s32(&sA[r0][ks + 8 + 2 * tq]);
                a[3] = ld_s32(&sA[r0 + 8][ks + 8 + 2 * tq]);
#pragma unroll
                for (int n = 0; n < BN / 8; ++n) {
                    unsigned b[2];
                    b[0] = ld_s32(&sB[n * 8 + g][ks + 2 * tq]);
                    b[1] = ld_s32(&sB[n * 8 + g][ks + 8 + 2 * tq]);
                    mma_bf16(acc[n], a, b);
                }
            }
            __syncthreads();
        }
    }
    // epilogue: rows w*16 + g (+8), columns n*8 + 2 tq (+1)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const long long vo = v0 + w * 16 + g + hh * 8;
        if (vo >= P.V) continue;
#pragma unroll
        for (int n = 0; n < BN / 8; ++n) {
            const int co = co0 + n * 8 + 2 * tq;
            float y0 = acc[n][2 * hh], y1 = acc[n][2 * hh + 1];
            if (RAW) {
                float2 *dst = reinterpret_cast<float2 *>(static_cast<float *>(P.Y) + vo * P.Cout + co);
                *dst = make_float2(y0, y1);
            } else {
                y0 = fmaxf(y0 + P.bias[co], 0.f);
                y1 = fmaxf(y1 + P.bias[co + 1], 0.f);
                __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(
                    static_cast<bf16 *>(P.Y) + vo * P.Cout + co);
                *dst = __floats2bfloat162_rn(y0, y1);
            }
        }
    }
}

// The same convolution on bricks of 4 x 4 x 8 cells (grid dimensions
// multiples of 4, 4, 8): per chunk of CK input channels the block loads the
// brick's 6 x 6 x 10 halo once and the chunk's weights of all 27 taps, then
// runs every tap's MMAs from shared memory (the plain kernel reloads the
// inputs for each tap).  32 output channels per block; each warp owns 32
// cells (two m16 tiles).
constexpr int HXB = 4, HYB = 4, HZB = 8;        // brick
constexpr int HCELLS = (HXB + 2) * (HYB + 2) * (HZB + 2);
constexpr int HBN = 32;

template <int CK_>
struct HaloSmem {
    bf16 h[HCELLS][CK_ + 8];
    bf16 w[27][HBN][CK_ + 8];
};

template <int CK_, bool RAW>
__global__ void __launch_bounds__(128) k_conv_halo(ConvArgs P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HaloSmem<CK_> &S = *reinterpret_cast<HaloSmem<CK_> *>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int bxn = P.nx / HXB, byn = P.ny / HYB;
    const int bz = blockIdx.x % (P.nz / HZB);
    const int by = (blockIdx.x / (P.nz / HZB)) % byn;
    const int bx = blockIdx.x / ((P.nz / HZB) * byn);
    (void)bxn;
    const int i0 = bx * HXB, j0 = by * HYB, k0 = bz * HZB;
    const int co0 = blockIdx.y * HBN;
    const int Cin = P.Ca + P.Cb;
    const long long nyz = (long long)P.ny * P.nz;
    const int hy = P.ny >> 1, hz = P.nz >> 1;
    // halo index of the rows this lane reads: cell q = 32 w + 16 m + g (+8)
    int hrow[2][2];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int q = 32 * w + 16 * m + g + 8 * hh;
            const int cx = q / (HYB * HZB), cy = (q / HZB) % HYB, cz = q % HZB;
            hrow[m][hh] = ((cx + 1) * (HYB + 2) + (cy + 1)) * (HZB + 2) + (cz + 1);
        }
    float acc[2][HBN / 8][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < HBN / 8; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
    constexpr int V16 = CK_ / 8;   // uint4 per cell row of the chunk
    for (int c0 = 0; c0 < Cin; c0 += CK_) {
        // halo of the chunk
        for (int e = t; e < HCELLS * V16; e += 128) {
            const int hc = e / V16, part = e % V16;
            const int hx = hc / ((HYB + 2) * (HZB + 2)), hyy = (hc / (HZB + 2)) % (HYB + 2),
                      hzz = hc % (HZB + 2);
            const int ii = i0 + hx - 1, jj = j0 + hyy - 1, kk = k0 + hzz - 1;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (ii >= 0 && ii < P.nx && jj >= 0 && jj < P.ny && kk >= 0 && kk < P.nz) {
                const bf16 *src;
                if (c0 < P.Ca)
                    src = P.A + ((long long)ii * nyz + (long long)jj * P.nz + kk) * P.Ca + c0;
                else
                    src = P.B + (((long long)(ii >> 1) * hy + (jj >> 1)) * hz + (kk >> 1)) * P.Cb +
                          (c0 - P.Ca);
                v = reinterpret_cast<const uint4 *>(src)[part];
            }
            *reinterpret_cast<uint4 *>(&S.h[hc][part * 8]) = v;
        }
        // weights of all taps for the chunk
        for (int e = t; e < 27 * HBN * V16; e += 128) {
            const int tap = e / (HBN * V16), co = (e / V16) % HBN, part = e % V16;
            const bf16 *src = P.Wt + ((long long)tap * P.Cout + co0 + co) * Cin + c0;
            *reinterpret_cast<uint4 *>(&S.w[tap][co][part * 8]) =
                reinterpret_cast<const uint4 *>(src)[part];
        }
        __syncthreads();
        for (int tap = 0; tap < 27; ++tap) {
            const int off = ((tap / 9 - 1) * (HYB + 2) + ((tap / 3) % 3 - 1)) * (HZB + 2) +
                            (tap % 3 - 1);
#pragma unroll
            for (int ks = 0; ks < CK_; ks += 16) {
                unsigned b[HBN / 8][2];
#pragma unroll
                for (int n = 0; n < HBN / 8; ++n) {
                    b[n][0] = ld_s32(&S.w[tap][n * 8 + g][ks + 2 * tq]);
                    b[n][1] = ld_s32(&S.w[tap][n * 8 + g][ks + 8 + 2 * tq]);
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    unsigned a[4];
                    const int r0 = hrow[m][0] + off, r1 = hrow[m][1] + off;
                    a[0] = ld_s32(&S.h[r0][ks + 2 * tq]);
                    a[1] = ld_s32(&S.h[r1][ks + 2 * tq]);
                    a[2] = ld_s32(&S.h[r0][ks + 8 + 2 * tq]);
                    a[3] = ld_s32(&S.h[r1][ks + 8 + 2 * tq]);
#pragma unroll
                    for (int n = 0; n < HBN / 8; ++n) mma_bf16(acc[m][n], a, b[n]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int q = 32 * w + 16 * m + g + 8 * hh;
            const int cx = q / (HYB * HZB), cy = (q / HZB) % HYB, cz = q % HZB;
            const long long vo = (long long)(i0 + cx) * nyz + (long long)(j0 + cy) * P.nz + k0 + cz;
#pragma unroll
            for (int n = 0; n < HBN / 8; ++n) {
                const int co = co0 + n * 8 + 2 * tq;
                float y0 = acc[m][n][2 * hh], y1 = acc[m][n][2 * hh + 1];
                if (RAW) {
                    *reinterpret_cast<float2 *>(static_cast<float *>(P.Y) + vo * P.Cout + co) =
                        make_float2(y0, y1);
                } else {
                    y0 = fmaxf(y0 + P.bias[co], 0.f);
                    y1 = fmaxf(y1 + P.bias[co + 1], 0.f);
                    *reinterpret_cast<__nv_bfloat162 *>(static_cast<bf16 *>(P.Y) + vo * P.Cout +
                                                        co) = __floats2bfloat162_rn(y0, y1);
                }
            }
        }
}

// ------------------------------------------------------ tcgen05 convolution
// The same convolution on the 5th-generation tensor cores: one block of 4
// warps per brick of 1 x 16 x 8 cells (M = 128 rows of the accumulator in
// tensor memory), NT output channels (N), 32 input channels per stage.  The
// stage's halo (3 x 18 x 10 cells) and weights sit in shared memory in the
// canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes), so every tap's A operand is the halo itself seen through a
// descriptor: a core matrix is 8 cells along z (consecutive 16-byte rows),
// the next 8 rows of M are the next y column (a fixed stride), the next 8
// channels of K the next channel plane (another fixed stride).  One thread
// issues the 54 MMAs of a stage (27 taps x 2 steps of K = 16) and commits
// them to an mbarrier that guards the buffers of the next stage.
constexpr int TCY = 16, TCZ = 8;                           // brick (x extent 1)
constexpr int TC_HX = 3, TC_HY = TCY + 2, TC_HZ = TCZ + 2;
constexpr int TC_HALO_BYTES = TC_HX * TC_HY * 4 * TC_HZ * 16;   // 34,560
constexpr unsigned long long kTcWaitNs = 2000000000ull;   // 2 s bound on one wait
// MMAs into one accumulator run one after another; the taps are dealt over
// TC_CHAINS accumulators (summed in the epilogue) so that independent MMAs
// keep the tensor pipe busy.
constexpr int TC_CHAINS = 4;

__host__ __device__ constexpr int tc_w_bytes(int NT) { return 27 * 4 * NT * 16; }
__host__ __device__ constexpr int tc_smem_bytes(int NT)
{
    return tc_w_bytes(NT) + TC_HALO_BYTES + 64;
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr >> 4) & 0x3fffu) |
           ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D,
// M = 128, N = NT.
__host__ __device__ constexpr unsigned tc_idesc(int NT)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NT >> 3) << 17) | (8u << 24);
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// try_wait suspends the thread until the phase completes or a short
// hardware time limit passes, so the loop polls without sleeping; the
// global timer, read every 64 misses, bounds the whole wait.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    unsigned long long t0 = 0;
    for (unsigned i = 0;; ++i) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if ((i & 63u) == 0) {
            unsigned long long now;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
            if (i == 0) t0 = now;
            else if (now - t0 > kTcWaitNs) return false;
        }
    }
}

// 16-byte asynchronous global -> shared copy (zero fill when !valid): the
// loads of a stage are all in flight together instead of one round trip
// per iteration.
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

__device__ __forceinline__ void tc_mma(unsigned dcol, unsigned long long ad, unsigned long long bd,
                                       unsigned idesc, unsigned acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(dcol), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}

template <int NT, bool RAW>
__global__ void __launch_bounds__(128, 1) k_conv_tc(ConvArgs P, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sw = smem;                                 // weights
    unsigned char *sh = smem + tc_w_bytes(NT);                // halo
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(sh + TC_HALO_BYTES);
    unsigned *tslot = reinterpret_cast<unsigned *>(sh + TC_HALO_BYTES + 8);
    int *sfail = reinterpret_cast<int *>(sh + TC_HALO_BYTES + 16);
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int nyb = P.ny / TCY, nzb = P.nz / TCZ;
    const int bz = blockIdx.x % nzb, by = (blockIdx.x / nzb) % nyb, bx = blockIdx.x / (nzb * nyb);
    const int i0 = bx, j0 = by * TCY, k0 = bz * TCZ;
    const int co0 = blockIdx.y * NT;
    const int Cin = P.Ca + P.Cb;
    const long long nyz = (long long)P.ny * P.nz;
    const int hy = P.ny >> 1, hz = P.nz >> 1;
    const unsigned bar = smem_u32(mbar);
    if (t == 0) {
        *sfail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(TC_CHAINS * NT) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    const unsigned idesc = tc_idesc(NT);
    const int nstage = Cin / 32;
    for (int st = 0; st < nstage; ++st) {
        const int c0 = st * 32;
        if (st > 0 && !mbar_wait(bar, (unsigned)((st - 1) & 1))) {
            *sfail = 1;
            atomicExch(err, 1);
        }
        __syncthreads();
        if (*sfail) break;
        // weights of the stage: [tap][kc][co][8 ci]
        const unsigned swa = smem_u32(sw), sha = smem_u32(sh);
        for (int e = t; e < 27 * 4 * NT; e += 128) {
            const int co = e % NT, kc = (e / NT) % 4, tap = e / (4 * NT);
            const bf16 *src = P.Wt + ((long long)tap * P.Cout + co0 + co) * Cin + c0 + kc * 8;
            cp_async16(swa + (unsigned)e * 16u, src, true);
        }
        // halo of the stage: [hx][hy][kc][hz][8 ci], zero outside the grid
        for (int e = t; e < TC_HX * TC_HY * 4 * TC_HZ; e += 128) {
            const int hzz = e % TC_HZ, kc = (e / TC_HZ) % 4, hyy = (e / (4 * TC_HZ)) % TC_HY,
                      hxx = e / (4 * TC_HZ * TC_HY);
            const int ii = i0 + hxx - 1, jj = j0 + hyy - 1, kk = k0 + hzz - 1;
            const bool in = ii >= 0 && ii < P.nx && jj >= 0 && jj < P.ny && kk >= 0 && kk < P.nz;
            const bf16 *src = P.A;     // any valid address when nothing is read
            if (in) {
                if (c0 < P.Ca)
                    src = P.A + ((long long)ii * nyz + (long long)jj * P.nz + kk) * P.Ca + c0 +
                          kc * 8;
                else
                    src = P.B + (((long long)(ii >> 1) * hy + (jj >> 1)) * hz + (kk >> 1)) * P.Cb +
                          (c0 - P.Ca) + kc * 8;
            }
            cp_async16(sha + (unsigned)e * 16u, src, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // descriptors of tap 0, step 0; the others differ only in the
            // start address field (16-byte units), so they are one add away
            const unsigned long long ad0 = tc_desc(smem_u32(sh), TC_HZ * 16, 4 * TC_HZ * 16);
            const unsigned long long bd0 = tc_desc(smem_u32(sw), NT * 16, 8 * 16);
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const int da = tap / 9, db = (tap / 3) % 3, dc = tap % 3;   // halo offsets 0..2
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2) {
                    const unsigned long long ad =
                        ad0 + (unsigned long long)(((da * TC_HY + db) * 4 + 2 * s2) * TC_HZ + dc);
                    const unsigned long long bd = bd0 + (unsigned long long)((tap * 4 + 2 * s2) * NT);
                    const unsigned acc = (st > 0 || tap >= TC_CHAINS || s2 > 0) ? 1u : 0u;
                    tc_mma(tmem + (unsigned)((tap % TC_CHAINS) * NT), ad, bd, idesc, acc);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar) : "memory");
        }
    }
    const bool failed_before = *sfail != 0;
    __syncthreads();
    if (!failed_before && !mbar_wait(bar, (unsigned)((nstage - 1) & 1))) {
        *sfail = 1;     // every thread that timed out marks it; read after the barrier
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!*sfail) {
        const int m = 32 * w + lane;             // accumulator row = cell of the brick
        const long long vo = (long long)i0 * nyz + (long long)(j0 + m / TCZ) * P.nz + k0 + m % TCZ;
#pragma unroll
        for (int half = 0; half < NT / 32; ++half) {
            unsigned r[32];
            float sum[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) sum[c] = 0.f;
            for (int ch = 0; ch < TC_CHAINS; ++ch) {
            const unsigned ta = tmem + ((unsigned)(32 * w) << 16) + (unsigned)(ch * NT + 32 * half);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                  "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                  "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                  "=r"(r[30]), "=r"(r[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < 32; ++c) sum[c] += __uint_as_float(r[c]);
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) r[c] = __float_as_uint(sum[c]);
            const int cb = co0 + 32 * half;
            if (RAW) {
                float *dst = static_cast<float *>(P.Y) + vo * P.Cout + cb;
#pragma unroll
                for (int c = 0; c < 32; c += 4)
                    *reinterpret_cast<float4 *>(dst + c) =
                        make_float4(__uint_as_float(r[c]), __uint_as_float(r[c + 1]),
                                    __uint_as_float(r[c + 2]), __uint_as_float(r[c + 3]));
            } else {
                bf16 *dst = static_cast<bf16 *>(P.Y) + vo * P.Cout + cb;
#pragma unroll
                for (int c = 0; c < 32; c += 8) {
                    __align__(16) __nv_bfloat162 o[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        o[q] = __floats2bfloat162_rn(
                            fmaxf(__uint_as_float(r[c + 2 * q]) + P.bias[cb + c + 2 * q], 0.f),
                            fmaxf(__uint_as_float(r[c + 2 * q + 1]) + P.bias[cb + c + 2 * q + 1],
                                  0.f));
                    *reinterpret_cast<uint4 *>(dst + c) = *reinterpret_cast<const uint4 *>(o);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(TC_CHAINS * NT) : "memory");
    }
}

// Weight-stationary blocks: each block takes nb consecutive bricks (up to
// 512 / NT, chosen per launch) and keeps a stage's weights in shared memory
// for all of them, with one FP32 accumulator per brick in tensor memory (nb
// x NT columns).  The bricks' halos stream through NBUF buffers: the next
// bricks' halos load while the tensor cores run the current brick's MMAs; a
// buffer is refilled once the MMAs that read it have committed.  Stage
// boundaries wait for the stage's last MMAs before the weights are
// replaced.  The fixed cost of a block (tensor-memory allocation, barrier
// set-up, the first copies, the epilogue's drain) is spread over its
// bricks: 8 bricks per block instead of 4 took 6 % off the 384^3 forward.
__host__ __device__ constexpr int tma_max_nb(int NT) { return 512 / NT; }

// TMA form of the weight-stationary convolution, for inputs at the
// output's resolution (a decoder's coarse input is doubled first).  The
// stage's weights come pre-arranged in global memory (one contiguous block
// per stage and tile of output channels) and arrive by bulk copies (only
// the planes and taps the stage uses); a brick's halo arrives as
// tensor-map box loads (8 channels x 10 z x 18 y x 3 x each, or 1 x for
// x1, cells outside the grid zero-filled by the copy engine).  Copies and MMAs complete on mbarriers, so one
// thread runs the whole producer/consumer loop: it keeps the copies of the
// next NBUF - 1 bricks in flight while the tensor cores work, and the
// other warps only join for the epilogue.  Halo layout: [8-channel plane]
// [x][y][z][8 ch], planes 128-byte aligned.
constexpr int TMA_PLANE = 8704;                         // 540 x 16 B padded to 128 B
constexpr int TMA_HALO = 4 * TMA_PLANE;

// The halo area holds tma_nbuf(NT) full buffers; a stage that loads fewer
// planes (k16 = 1) or one x-plane (x1) cuts it into more, smaller buffers
// (up to TMA_MAXBUF), so that more bricks' copies are in flight.
__host__ __device__ constexpr int tma_nbuf(int NT) { return NT == 32 ? 4 : 3; }
constexpr int TMA_MAXBUF = 16;
constexpr int TMA_PLANE_X1 = 2944;                      // 180 x 16 B padded to 128 B
__host__ __device__ constexpr int tma_smem_bytes(int NT)
{
    return tc_w_bytes(NT) + tma_nbuf(NT) * TMA_HALO + 16 * TMA_MAXBUF + 128 + 128;
}

template <int NT, bool RAW>
__global__ void __launch_bounds__(128, 1)
k_conv_tma(ConvArgs P, const __grid_constant__ CUtensorMap tmA,
           const __grid_constant__ CUtensorMap tmB, const bf16 *__restrict__ Wtc, int nbricks,
           int nb, int *err)
{
    // plane stride, buffer size and buffer count of this launch
    const int PLs = P.x1 ? TMA_PLANE_X1 : TMA_PLANE;
    const int HB = 2 * P.k16 * PLs;
    const int NBUF = min(TMA_MAXBUF, tma_nbuf(NT) * TMA_HALO / HB);
    extern __shared__ __align__(1024) unsigned char smem_tma[];
    const unsigned raw0 = smem_u32(smem_tma);
    const unsigned pad = ((raw0 + 127u) & ~127u) - raw0;
    unsigned char *smem = smem_tma + pad;
    unsigned char *tail = smem + tc_w_bytes(NT) + tma_nbuf(NT) * TMA_HALO;
    unsigned *tslot = reinterpret_cast<unsigned *>(tail + 16 * TMA_MAXBUF);
    int *sfail = reinterpret_cast<int *>(tail + 16 * TMA_MAXBUF + 4);
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int nyb = P.ny / TCY, nzb = P.nz / TCZ;
    const int b0 = blockIdx.x * nb;
    const int nbv = min(nb, nbricks - b0);
    const int nst = (P.Ca + P.Cb) / 32;     // stages of the first input, then of the second
    const int U = nst * nbv;
    const int nnt = P.Cout / NT;
    const int co0 = blockIdx.y * NT;
    const unsigned swa = smem_u32(smem), sha0 = swa + (unsigned)tc_w_bytes(NT);
    const unsigned ldb0 = smem_u32(tail), mmb0 = ldb0 + 8u * NBUF;   // NBUF load + NBUF MMA barriers
    if (t == 0) {
        *sfail = 0;
        for (int q = 0; q < 2 * NBUF; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ldb0 + 8u * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];"
                     :: "l"(reinterpret_cast<unsigned long long>(&tmA)) : "memory");
        if (P.Cb > 0)
            asm volatile("prefetch.tensormap [%0];"
                         :: "l"(reinterpret_cast<unsigned long long>(&tmB)) : "memory");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    constexpr int CH = 1;       // accumulator chains per brick (more did not help)

    if (t == 0) {
        const unsigned idesc = tc_idesc(NT);
        // unit u: stage u / nbv, brick u % nbv, buffer u % NBUF (its k-th
        // use, k = u / NBUF, completes phase k of that buffer's barriers)
        int issued = 0;      // units whose copies have been issued (in order)
        auto issue = [&](int u) {
            issued = u + 1;
            const int st = u / nbv, bb = b0 + u % nbv, c0 = st * 32;
            const int bz = bb % nzb, by = (bb / nzb) % nyb, bx = bb / (nzb * nyb);
            const unsigned buf = (unsigned)(u % NBUF);
            const unsigned lb = ldb0 + 8u * buf;
            const unsigned sha = sha0 + buf * (unsigned)HB;
            const bool wload = (u % nbv) == 0;
            // x1: the halo is the brick's own x-plane only (180 rows per box)
            // the stage's weights [8-channel plane][tap][co][8 ch]: all of
            // them, or for a half-filled stage (k16 = 1) the first two
            // planes, and with x1 only the taps 9..17 of each
            const bool wall = P.k16 == 2 && !P.x1;
            const int ntap = P.x1 ? 9 : 27, tap0 = P.x1 ? 9 : 0;
            const unsigned wrun = (unsigned)(ntap * NT * 16);
            const unsigned wbytes = wall ? (unsigned)tc_w_bytes(NT) : 2u * (unsigned)P.k16 * wrun;
            const unsigned tx = 2u * (unsigned)P.k16 * (P.x1 ? 180u : 540u) * 16u +
                                (wload ? wbytes : 0u);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(lb), "r"(tx) : "memory");
            if (wload) {
                const bf16 *src = Wtc + (size_t)(st * nnt + blockIdx.y) * (4 * 27 * NT * 8);
                if (wall) {
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                        :: "r"(swa), "l"(src), "r"((unsigned)tc_w_bytes(NT)), "r"(lb) : "memory");
                } else {
                    for (int kc = 0; kc < 2 * P.k16; ++kc) {
                        const unsigned off = (unsigned)((kc * 27 + tap0) * NT * 16);
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                            :: "r"(swa + off), "l"(reinterpret_cast<const unsigned char *>(src) + off),
                               "r"(wrun), "r"(lb) : "memory");
                    }
                }
            }
            const bool first_input = c0 < P.Ca;
            const unsigned long long map = reinterpret_cast<unsigned long long>(first_input ? &tmA : &tmB);
            const int cc = first_input ? c0 : c0 - P.Ca;
            for (int kc = 0; kc < 2 * P.k16; ++kc)
                asm volatile(
                    "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                    :: "r"(sha + (unsigned)(kc * PLs)), "l"(map),
                       "r"(cc + 8 * kc), "r"(bz * TCZ - 1), "r"(by * TCY - 1),
                       "r"(P.x1 ? bx : bx - 1), "r"(lb)
                    : "memory");
        };
        auto wait_bar = [&](unsigned base, int u) -> bool {
            return mbar_wait(base + 8u * (unsigned)(u % NBUF), (unsigned)((u / NBUF) & 1));
        };
        bool ok = true;
        // prologue: the first stage's first NBUF - 1 bricks
        for (int v = 0; v < NBUF - 1 && v < nbv && v < U; ++v) issue(v);
        for (int u = 0; u < U && ok; ++u) {
            const int st = u / nbv;
            if (!wait_bar(ldb0, u)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned hbase = sha0 + (unsigned)(u % NBUF) * (unsigned)HB;
            const unsigned long long ad0 = tc_desc(hbase, (unsigned)PLs, TC_HZ * 16);
            const unsigned long long bd0 = tc_desc(swa, 27 * NT * 16, 8 * 16);
            const unsigned dbase = tmem + (unsigned)((u % nbv) * CH * NT);
            const bool first = st == 0;
            // with x1 only the taps 9..17 (x offset 0) run; the first CH of
            // them start the accumulator chains
            const int t0 = P.x1 ? 9 : 0;
            if (P.k16 == 2) {
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int da = tap / 9, db = (tap / 3) % 3, dc = tap % 3;
                    if (P.x1 && da != 1) continue;
                    const unsigned long long ao =
                        (unsigned long long)(((P.x1 ? 0 : da) * TC_HY + db) * TC_HZ + dc);
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2)
                        tc_mma(dbase + (unsigned)((tap % CH) * NT),
                               ad0 + ao + (unsigned long long)(2 * s2 * (PLs / 16)),
                               bd0 + (unsigned long long)((2 * s2 * 27 + tap) * NT), idesc,
                               (!first || tap >= t0 + CH || s2 > 0) ? 1u : 0u);
                }
            } else {
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const int da = tap / 9, db = (tap / 3) % 3, dc = tap % 3;
                    if (P.x1 && da != 1) continue;
                    const unsigned long long ao =
                        (unsigned long long)(((P.x1 ? 0 : da) * TC_HY + db) * TC_HZ + dc);
                    tc_mma(dbase + (unsigned)((tap % CH) * NT), ad0 + ao,
                           bd0 + (unsigned long long)(tap * NT), idesc,
                           (!first || tap >= t0 + CH) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mmb0 + 8u * (unsigned)(u % NBUF)) : "memory");
            // with this brick's MMAs queued, refill the buffer the previous
            // brick read (unit u + NBUF - 1 of the same stage): the tensor
            // cores never wait for the issuing thread
            const int v = u + NBUF - 1;
            if (v < U && v / nbv == st) {
                if (v >= NBUF && !wait_bar(mmb0, v - NBUF)) { ok = false; break; }
                issue(v);
            }
            // stage boundary: replace the weights once every MMA of the stage
            // has completed, then refill the pipeline
            if (u + 1 < U && (u + 1) % nbv == 0) {
                if (!wait_bar(mmb0, u)) { ok = false; break; }
                for (int q = u + 1; q < u + NBUF && q < U && q / nbv == (u + 1) / nbv; ++q)
                    issue(q);
            }
        }
        if (ok && U > 0 && !wait_bar(mmb0, U - 1)) ok = false;
        if (!ok) {
            *sfail = 1;
            atomicExch(err, 1);
            // copies still in flight target this block's shared memory:
            // wait (bounded) for the last one of each buffer
            for (int q = max(0, issued - NBUF); q < issued; ++q) wait_bar(ldb0, q);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!*sfail) {
        // Each warp holds 32 cells of a brick: one y row of 8 z cells per 8
        // lanes.  A cell's outputs pass through the (now idle) halo buffers
        // so that each store instruction writes whole 64- or 128-byte cell
        // rows instead of one 16-byte piece of 32 cells.  Chunk slots are
        // XOR-swizzled so that neither side has bank conflicts.
        const long long nyz = (long long)P.ny * P.nz;
        uint4 *stg = reinterpret_cast<uint4 *>(smem + tc_w_bytes(NT)) + w * 256;   // 4 KB per warp
        for (int b = 0; b < nbv; ++b) {
            const int bb = b0 + b;
            const int bz = bb % nzb, by = (bb / nzb) % nyb, bx = bb / (nzb * nyb);
            // cell of warp-local index c: row c >> 3 (y), z = c & 7
            const long long vrow = (long long)bx * nyz + (long long)(by * TCY + 4 * w) * P.nz +
                                   bz * TCZ;
            const long long vo = vrow + (long long)(lane >> 3) * P.nz + (lane & 7);
#pragma unroll
            for (int half = 0; half < NT / 32; ++half) {
                unsigned r[32];
                const unsigned ta = tmem + ((unsigned)(32 * w) << 16) +
                                    (unsigned)(b * CH * NT + 32 * half);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                      "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                      "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                      "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                const int cb = co0 + 32 * half;
                if (RAW) {
                    // FP32: 8 chunks of 16 bytes per cell
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        stg[lane * 8 + (q ^ (lane & 7))] =
                            make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
                    __syncwarp();
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        const int c = 4 * s + (lane >> 3), q = lane & 7;
                        float *dst = static_cast<float *>(P.Y) +
                                     (vrow + (long long)(c >> 3) * P.nz + (c & 7)) * P.Cout + cb + 4 * q;
                        *reinterpret_cast<uint4 *>(dst) = stg[c * 8 + (q ^ (c & 7))];
                    }
                    __syncwarp();
                } else {
                    float hzv = P.hz ? *P.hb : 0.f;
                    __align__(16) __nv_bfloat162 o[16];
#pragma unroll
                    for (int c = 0; c < 32; c += 2)
                        o[c / 2] = __floats2bfloat162_rn(
                            fmaxf(__uint_as_float(r[c]) + P.bias[cb + c], 0.f),
                            fmaxf(__uint_as_float(r[c + 1]) + P.bias[cb + c + 1], 0.f));
                    if (P.hz) {      // the head's sum, in channel order
#pragma unroll
                        for (int c = 0; c < 16; ++c) {
                            const float2 f = __bfloat1622float2(o[c]);
                            hzv = fmaf(P.hw[2 * c], f.x, hzv);
                            hzv = fmaf(P.hw[2 * c + 1], f.y, hzv);
                        }
                        P.hz[vo] = hzv;
                    } else {
                        // BF16: 4 chunks of 16 bytes per cell
                        const uint4 *ov = reinterpret_cast<const uint4 *>(o);
#pragma unroll
                        for (int q = 0; q < 4; ++q) stg[lane * 4 + (q ^ ((lane >> 1) & 3))] = ov[q];
                        __syncwarp();
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            const int c = 8 * s + (lane >> 2), q = lane & 3;
                            bf16 *dst = static_cast<bf16 *>(P.Y) +
                                        (vrow + (long long)(c >> 3) * P.nz + (c & 7)) * P.Cout + cb + 8 * q;
                            *reinterpret_cast<uint4 *>(dst) = stg[c * 4 + (q ^ ((c >> 1) & 3))];
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(512) : "memory");
    }
}

// Nearest doubling: Y[v][c] = X[parent(v)][c] for a fine grid nx x ny x nz
// (16-byte copies; C / 8 = 2^qs groups of 8 channels): fine row (i, j) on
// blockIdx.x, (k, group) on blockIdx.y x blockDim.x.
__global__ void k_upsample(const bf16 *__restrict__ X, int nx, int ny, int nz, int C, int qs,
                           bf16 *__restrict__ Y)
{
    const int q = C >> 3;
    const int row = blockIdx.x, i = row / ny, j = row - i * ny;
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= nz * q) return;
    const int k = e >> qs, part = e & (q - 1);
    const long long u = ((long long)(i >> 1) * (ny >> 1) + (j >> 1)) * (nz >> 1) + (k >> 1);
    reinterpret_cast<uint4 *>(Y + ((long long)row * nz + k) * C)[part] =
        reinterpret_cast<const uint4 *>(X + u * C)[part];
}

// Weights [27][Cout][Cin] -> the TMA form's layout: per stage of 32 input
// channels and tile of NT output channels, [8-channel plane][tap][co][8].
__global__ void k_pack_tc(const bf16 *__restrict__ W, int Cout, int Cin, int NT,
                          bf16 *__restrict__ out)
{
    const long long n = 27ll * Cout * Cin;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int tap = (int)(e / ((long long)Cout * Cin));
    const int co = (int)((e / Cin) % Cout);
    const int ci = (int)(e % Cin);
    const int st = ci / 32, kc = (ci % 32) / 8, j = ci % 8;
    const int nt = co / NT, col = co % NT, nnt = Cout / NT;
    out[((((long long)(st * nnt + nt) * 4 + kc) * 27 + tap) * NT + col) * 8 + j] = W[e];
}

// Weight gradient of a conv3: dW[tap][co][ci] = sum over cells v of
// dZ[v][co] X[v + tap][ci] (X the concatenated input).  M = co (64 per
// block), N = ci (32 per block), K = cells in stages of 32, split over
// chunks of cells_per_block cells; each chunk writes its own partial
// dW (part[chunk][tap][co][ci]) and k_sum_parts4 adds the chunks in order,
// so the result does not depend on the order the blocks run in.
struct WgradArgs {
    int nx, ny, nz;
    long long V;
    const bf16 *A;
    int Ca;
    const bf16 *B;
    int Cb;
    const bf16 *dZ;      // [V][Cout]
    int Cout;
    float *part;         // [chunks][27][Cout][Cin]
    long long cells_per_block;
};

constexpr int WK = 32;           // cells per stage
constexpr int WROW = WK + 8;

__global__ void __launch_bounds__(128) k_wgrad(WgradArgs P)
{
    __shared__ __align__(16) bf16 sZ[64][WROW];   // [co][cell]
    __shared__ __align__(16) bf16 sX[32][WROW];   // [ci][cell]
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int Cin = P.Ca + P.Cb;
    const int nci = Cin / 32;
    const int tap = blockIdx.y / nci, ci0 = (blockIdx.y % nci) * 32;
    const int co0 = blockIdx.z * 64;
    const int da = tap / 9 - 1, db = (tap / 3) % 3 - 1, dc = tap % 3 - 1;
    const long long nyz = (long long)P.ny * P.nz;
    const int hy = P.ny >> 1, hz = P.nz >> 1;
    const long long vb = (long long)blockIdx.x * P.cells_per_block;
    const long long ve = min(vb + P.cells_per_block, P.V);
    float acc[4][4];
#pragma unroll
    for (int n = 0; n < 4; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    const int r = t >> 2, q = t & 3;     // staged cell and quarter
    for (long long s0 = vb; s0 < ve; s0 += WK) {
        const long long v = s0 + r;
        // dZ[v][co0 + 16q .. +16] -> sZ[.][r] (zero beyond Cout when Cout = 32)
        {
            __align__(16) bf16 z[16];
            if (v < ve && co0 + q * 16 < P.Cout) {
                const uint4 *s4 = reinterpret_cast<const uint4 *>(P.dZ + v * P.Cout + co0 + q * 16);
                reinterpret_cast<uint4 *>(z)[0] = s4[0];
                reinterpret_cast<uint4 *>(z)[1] = s4[1];
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) z[e] = __float2bfloat16(0.f);
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) sZ[q * 16 + e][r] = z[e];
        }
        // X[v + tap][ci0 + 8q .. +8] -> sX[.][r]
        {
            __align__(16) bf16 x[8];
            bool ok = false;
            long long src = 0;
            int ii = 0, jj = 0, kk = 0;
            if (v < ve) {
                const int i = (int)(v / nyz);
                const long long rem = v - (long long)i * nyz;
                const int j = (int)(rem / P.nz);
                const int k = (int)(rem - (long long)j * P.nz);
                ii = i + da;
                jj = j + db;
                kk = k + dc;
                ok = ii >= 0 && ii < P.nx && jj >= 0 && jj < P.ny && kk >= 0 && kk < P.nz;
            }
            if (ok) {
                const int c = ci0 + q * 8;
                const bf16 *p;
                if (c < P.Ca) {
                    src = (long long)ii * nyz + (long long)jj * P.nz + kk;
                    p = P.A + src * P.Ca + c;
                } else {
                    src = ((long long)(ii >> 1) * hy + (jj >> 1)) * hz + (kk >> 1);
                    p = P.B + src * P.Cb + (c - P.Ca);
                }
                reinterpret_cast<uint4 *>(x)[0] = *reinterpret_cast<const uint4 *>(p);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = __float2bfloat16(0.f);
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) sX[q * 8 + e][r] = x[e];
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < WK; ks += 16) {
            unsigned a[4];
            const int r0 = w * 16 + g;
            a[0] = ld_s32(&sZ[r0][ks + 2 * tq]);
            a[1] = ld_s32(&sZ[r0 + 8][ks + 2 * tq]);
            a[2] = ld_s32(&sZ[r0][ks + 8 + 2 * tq]);
            a[3] = ld_s32(&sZ[r0 + 8][ks + 8 + 2 * tq]);
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                unsigned b[2];
                b[0] = ld_s32(&sX[n * 8 + g][ks + 2 * tq]);
                b[1] = ld_s32(&sX[n * 8 + g][ks + 8 + 2 * tq]);
                mma_bf16(acc[n], a, b);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int co = co0 + w * 16 + g + hh * 8;
        if (co >= P.Cout) continue;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const int ci = ci0 + n * 8 + 2 * tq;
            float *d = P.part + (((long long)blockIdx.x * 27 + tap) * P.Cout + co) * Cin + ci;
            d[0] = acc[n][2 * hh];
            d[1] = acc[n][2 * hh + 1];
        }
    }
}

// ------------------------------------------------ tcgen05 weight gradient
// dW[tap][co][ci] = sum over cells v of dZ[v][co] X[v + tap][ci] on the
// 5th-generation tensor cores, for levels that tile by bricks of 1 x 16 x 8
// cells.  Per tap this is D[m][n] += sum over cells of P[cell][m] Q[cell][n]
// (K = cells): one operand gives the 128 rows of D (M, zero channels pad it
// to 128), the other its N columns.  Both operands sit in shared memory
// MN-major without swizzle - a core matrix is 8 cells along z (16-byte
// rows) by 8 channels - so the tiles keep the activations' channels-last
// layout and nothing is transposed.  The dZ brick is [y][channel group][z][8]
// and the input's halo [hx][hy][channel group][hz][8], as in the forward
// kernel, so every tap's operand is the same halo seen from another start
// address.  Rows are output channels when Cout >= Cin (encoder layers), else
// a 128-channel tile of the input (decoder layers, whose input is the skip
// and the doubled coarse tensor).  A block takes a chunk of consecutive
// bricks and a group of taps whose accumulators fill the tensor memory (512
// / N taps of N columns); one thread issues each brick's MMAs (8 per tap, K
// = 16 cells = two z-columns of the brick) once its tiles are staged, and
// the block writes its partial dW of those taps at the end, summed over the
// chunks in order afterwards.
constexpr int WT_KCM = 16;                                   // 128 M channels
constexpr int WT_DZ_BYTES = TCY * WT_KCM * TCZ * 16;          // 32,768
constexpr int WT_HALO_BYTES = TC_HX * TC_HY * WT_KCM * TC_HZ * 16;   // 138,240
// buffer sets (one or two, as they fit) and the barriers in the last 64 bytes
constexpr int WT_SMEM = 227 * 1024;
static_assert(WT_DZ_BYTES + WT_HALO_BYTES + 1024 <= WT_SMEM, "wgrad smem layout");

struct WgradTcArgs {
    int nx, ny, nz;
    const bf16 *A;       // input, skip part [V][Ca]
    int Ca;
    const bf16 *B;       // coarse part at half resolution [V / 8][Cb], or NULL
    int Cb;
    const bf16 *dZ;      // [V][Cout]
    int Cout;
    float *part;         // [chunks][27][Cout][Cin]
    int rows_co;         // 1: rows of D are output channels; 0: input channels
    int N;               // columns of D per tap
    int taps;            // taps per block (tap group)
    int bricks_per_chunk;
    int nbricks;
};

// Instruction descriptor of kind::f16 with both operands MN-major: BF16 A
// and B, FP32 D, M = 128, N.
__host__ __device__ constexpr unsigned wt_idesc(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
           ((unsigned)(N >> 3) << 17) | (8u << 24);
}

__device__ __forceinline__ int ilog2(int v)
{
    return 31 - __clz(v);
}

__global__ void __launch_bounds__(128, 1) k_wgrad_tc(WgradTcArgs P, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int Cin = P.Ca + P.Cb;
    const int nyb = P.ny / TCY, nzb = P.nz / TCZ;
    const long long nyz = (long long)P.ny * P.nz;
    const int hy = P.ny >> 1, hz = P.nz >> 1;
    const int chunk = blockIdx.x;
    const int tap0 = blockIdx.y * P.taps;
    const int ntap = min(P.taps, 27 - tap0);
    const int ci0 = P.rows_co ? 0 : blockIdx.z * 128;   // first input channel of the rows
    // channel groups (8 channels) in the layout and staged: the operand that
    // gives the 128 rows of D is laid out with 16 groups, the ones past its
    // channels zero (written once); the other has exactly its channels
    const int kcz = P.rows_co ? WT_KCM : P.Cout / 8;
    const int kch = P.rows_co ? Cin / 8 : WT_KCM;
    const int gz = P.Cout / 8;
    const int gh = P.rows_co ? Cin / 8 : min(WT_KCM, (Cin - ci0) / 8);
    const int lgz = ilog2(gz), lgh = ilog2(gh);          // both powers of two
    const int dz_bytes = TCY * kcz * TCZ * 16;
    const int h_bytes = TC_HX * TC_HY * kch * TC_HZ * 16;
    const int set_bytes = (dz_bytes + h_bytes + 1023) & ~1023;
    const int nbuf = 2 * set_bytes + 1024 <= WT_SMEM ? 2 : 1;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(smem + WT_SMEM - 64);
    unsigned *tslot = reinterpret_cast<unsigned *>(smem + WT_SMEM - 32);
    int *sfail = reinterpret_cast<int *>(smem + WT_SMEM - 28);
    const int b0 = chunk * P.bricks_per_chunk;
    const int b1 = min(P.nbricks, b0 + P.bricks_per_chunk);
    const int nb = b1 - b0;
    if (t == 0) {
        *sfail = 0;
        for (int q = 0; q < 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar + q)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero the padding groups of every buffer set once
    for (int q = 0; q < nbuf; ++q) {
        uint4 *sz = reinterpret_cast<uint4 *>(smem + q * set_bytes);
        uint4 *sh = reinterpret_cast<uint4 *>(smem + q * set_bytes + dz_bytes);
        if (gz < kcz)
            for (int e = t; e < TCY * kcz * TCZ; e += 128)
                if (((e / TCZ) % kcz) >= gz) sz[e] = make_uint4(0u, 0u, 0u, 0u);
        if (gh < kch)
            for (int e = t; e < TC_HX * TC_HY * kch * TC_HZ; e += 128)
                if (((e / TC_HZ) % kch) >= gh) sh[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    const unsigned idesc = wt_idesc(P.N);

    // stages brick b into buffer set q (cp.async, one group committed)
    auto stage = [&](int b, int q) {
        const int bz = b % nzb, by = (b / nzb) % nyb, bx = b / (nzb * nyb);
        const int i0 = bx, j0 = by * TCY, k0 = bz * TCZ;
        const unsigned sza = smem_u32(smem + q * set_bytes), sha = sza + (unsigned)dz_bytes;
        // dZ brick: [y][group][z][8 channels]; item e = ((y * gz) + g) * 8 + z
        for (int e = t; e < TCY * gz * TCZ; e += 128) {
            const int z = e & 7, g = (e >> 3) & (gz - 1), y = e >> (3 + lgz);
            const bf16 *src = P.dZ + ((long long)i0 * nyz + (long long)(j0 + y) * P.nz + k0 + z) *
                                         P.Cout + g * 8;
            cp_async16(sza + (unsigned)(((y * kcz + g) * TCZ + z) * 16), src, true);
        }
        // halo: [hx][hy][group][hz][8 channels], zero outside the grid;
        // item e = ((row * gh) + g) * 10 + hz with row = hx * 18 + hy
        for (int e = t; e < TC_HX * TC_HY * gh * TC_HZ; e += 128) {
            const int hzz = e % TC_HZ, rest = e / TC_HZ;
            const int g = rest & (gh - 1), row = rest >> lgh;
            const int hyy = row % TC_HY, hxx = row / TC_HY;
            const int ii = i0 + hxx - 1, jj = j0 + hyy - 1, kk = k0 + hzz - 1;
            const int c = ci0 + g * 8;
            const bool in = ii >= 0 && ii < P.nx && jj >= 0 && jj < P.ny && kk >= 0 && kk < P.nz;
            const bf16 *src = P.A;
            if (in) {
                if (c < P.Ca)
                    src = P.A + ((long long)ii * nyz + (long long)jj * P.nz + kk) * P.Ca + c;
                else
                    src = P.B + (((long long)(ii >> 1) * hy + (jj >> 1)) * hz + (kk >> 1)) * P.Cb +
                          (c - P.Ca);
            }
            cp_async16(sha + (unsigned)((((row * kch) + g) * TC_HZ + hzz) * 16), src, in);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // brick j of the chunk uses buffer set j % nbuf; its MMAs commit to
    // mbarrier j % 2 (the j / 2-th completion of that barrier)
    auto wait_mma = [&](int j) -> bool {
        return mbar_wait(smem_u32(mbar + (j & 1)), (unsigned)((j >> 1) & 1));
    };
    if (nb > 0) stage(b0, 0);
    for (int j = 0; j < nb; ++j) {
        const int q = j % nbuf;
        if (nbuf == 2) {
            // the other set is free once brick j - 1's MMAs have completed
            if (j >= 1 && !wait_mma(j - 1)) {
                *sfail = 1;
                atomicExch(err, 1);
            }
            __syncthreads();
            if (*sfail) break;
            if (j + 1 < nb) {
                stage(b0 + j + 1, (j + 1) % 2);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sza = smem_u32(smem + q * set_bytes), sha = sza + (unsigned)dz_bytes;
            // MN stride (SBO) between channel groups, K stride (LBO) between
            // the two z-columns of a K step
            const unsigned long long dz0 = tc_desc(sza, kcz * TCZ * 16, TCZ * 16);
            const unsigned long long dh0 = tc_desc(sha, kch * TC_HZ * 16, TC_HZ * 16);
            for (int jt = 0; jt < ntap; ++jt) {
                const int tap = tap0 + jt;
                const int da = tap / 9, db = (tap / 3) % 3, dc = tap % 3;
#pragma unroll
                for (int s2 = 0; s2 < TCY / 2; ++s2) {
                    // start addresses in 16-byte units
                    const unsigned long long oz = (unsigned long long)(2 * s2 * kcz * TCZ);
                    const unsigned long long oh =
                        (unsigned long long)(((da * TC_HY + 2 * s2 + db) * kch) * TC_HZ + dc);
                    const unsigned long long ad = P.rows_co ? dz0 + oz : dh0 + oh;
                    const unsigned long long bd = P.rows_co ? dh0 + oh : dz0 + oz;
                    const unsigned acc = (j > 0 || s2 > 0) ? 1u : 0u;
                    tc_mma(tmem + (unsigned)(jt * P.N), ad, bd, idesc, acc);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mbar + (j & 1))) : "memory");
        }
        if (nbuf == 1) {
            // one buffer set: the next brick's copies wait for these MMAs
            if (!wait_mma(j)) {
                *sfail = 1;
                atomicExch(err, 1);
            }
            __syncthreads();
            if (*sfail) break;
            if (j + 1 < nb) stage(b0 + j + 1, 0);
        }
    }
    const bool failed_before = *sfail != 0;
    __syncthreads();
    if (!failed_before && nb > 0 && nbuf == 2 && !wait_mma(nb - 1)) {
        *sfail = 1;
        atomicExch(err, 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!*sfail && nb > 0) {
        const int m = 32 * w + lane;                    // row of D
        for (int jt = 0; jt < ntap; ++jt) {
            const int tap = tap0 + jt;
            for (int n0 = 0; n0 < P.N; n0 += 32) {
                unsigned r[32];
                const unsigned ta = tmem + ((unsigned)(32 * w) << 16) + (unsigned)(jt * P.N + n0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                      "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                      "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                      "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float *base = P.part + ((long long)chunk * 27 + tap) * P.Cout * Cin;
                if (P.rows_co) {
                    if (m < P.Cout) {
                        float4 *d = reinterpret_cast<float4 *>(base + (long long)m * Cin + n0);
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            d[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                               __uint_as_float(r[4 * q + 2]),
                                               __uint_as_float(r[4 * q + 3]));
                    }
                } else if (ci0 + m < Cin) {
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        base[(long long)(n0 + q) * Cin + ci0 + m] = __uint_as_float(r[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(512) : "memory");
    }
}

// Fixed-order reductions of per-block partial gradients: out[i] = the sum
// over b = 0, 1, ... of part[b][i] (n entries per part), always added in
// the same order, so the result does not depend on how the blocks ran.

// Few entries and many parts: block i sums entry i, each
// thread the parts t, t + 256, ... in that order, then the threads in a
// fixed tree.
__global__ void __launch_bounds__(256) k_sum_parts_tree(const float *__restrict__ part,
                                                        int nparts, int n,
                                                        float *__restrict__ out)
{
    __shared__ float s_p[256];
    const int i = blockIdx.x;
    float s = 0.f;
    for (int b = threadIdx.x; b < nparts; b += 256) s += part[(long long)b * n + i];
    s_p[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s_p[threadIdx.x] += s_p[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = s_p[0];
}

// Many entries: n4 groups of 4 (n = 4 n4), 16-byte loads, eight
// parts' loads in flight at a time, each entry's sum still taken in part
// order.
__global__ void k_sum_parts4(const float4 *__restrict__ part, int nparts, long long n4,
                             float4 *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    int b = 0;
    for (; b + 8 <= nparts; b += 8) {
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldg(part + (long long)(b + q) * n4 + i);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            s.x += v[q].x;
            s.y += v[q].y;
            s.z += v[q].z;
            s.w += v[q].w;
        }
    }
    for (; b < nparts; ++b) {
        const float4 v = __ldg(part + (long long)b * n4 + i);
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
    }
    out[i] = s;
}

// ------------------------------------------------------------ small kernels
// x (F planes of the full grid NX x NY x NZ, FP32) cropped at (ox, oy, oz)
// to nx x ny x nz -> X0 [cell][32] bf16: channel f = feature f, or with
// fold channel dx F + f = feature f of the x neighbour dx - 1; unused
// channels zero.  One thread per cell: coalesced plane reads, four 16-byte
// stores.
template <int FF>     // FF > 0: F = FF known at compile time (the fold's indices fold away)
__global__ void k_pack_input(const float *__restrict__ x, int Frt, int NX, int NY, int NZ,
                             int ox, int oy, int oz, int nx, int ny, int nz, bool fold,
                             bf16 *__restrict__ X0)
{
    const int F = FF > 0 ? FF : Frt;
    // row (i, j) on blockIdx.x, z on blockIdx.y x blockDim.x
    const int row = blockIdx.x, i = row / ny, j = row - i * ny;
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= nz) return;
    const long long v = (long long)row * nz + k;
    const long long G = (long long)NX * NY * NZ;
    const long long src = ((long long)(i + ox) * NY + (j + oy)) * NZ + (k + oz);
    __align__(16) bf16 c[kInPad];
    if (fold) {
        // channel dx F + f: feature f of the cell at x offset dx - 1 (zero
        // outside the crop, as the convolution pads)
#pragma unroll
        for (int q = 0; q < kInPad; ++q) {
            const int dx = q / F, f = q - dx * F, ii = i + dx - 1;
            c[q] = __float2bfloat16(dx < 3 && ii >= 0 && ii < nx
                                        ? x[f * G + src + (long long)(dx - 1) * NY * NZ]
                                        : 0.f);
        }
    } else {
#pragma unroll
        for (int q = 0; q < kInPad; ++q) c[q] = __float2bfloat16(q < F ? x[q * G + src] : 0.f);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(X0 + v * kInPad);
#pragma unroll
    for (int q = 0; q < kInPad / 8; ++q) dst[q] = reinterpret_cast<const uint4 *>(c)[q];
}

// 2x2x2 mean pooling of [cell][C] bf16 at (nx, ny, nz) -> half resolution.
// One thread per coarse cell and group of 8 channels (C / 8 = 2^qs groups):
// output row (i, j) on blockIdx.x, (k, group) on blockIdx.y x blockDim.x.
// Each channel sums its 8 children in the same order as before, then
// scales by 1/8.
__global__ void k_pool(const bf16 *__restrict__ X, int nx, int ny, int nz, int C, int qs,
                       bf16 *__restrict__ Y)
{
    const int hy = ny >> 1, hz = nz >> 1, q = C >> 3;
    const int row = blockIdx.x, i = row / hy, j = row - i * hy;
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= hz * q) return;
    const int k = e >> qs, part = e & (q - 1);
    float s[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) s[c] = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const long long v = ((long long)(2 * i + (d >> 2)) * ny + 2 * j + ((d >> 1) & 1)) * nz +
                            2 * k + (d & 1);
        const uint4 w = reinterpret_cast<const uint4 *>(X + v * C)[part];
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float2 f = __bfloat1622float2(h[c]);
            s[2 * c] += f.x;
            s[2 * c + 1] += f.y;
        }
    }
    __align__(16) __nv_bfloat162 o[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = __floats2bfloat162_rn(s[2 * c] * 0.125f, s[2 * c + 1] * 0.125f);
    reinterpret_cast<uint4 *>(Y + ((long long)row * hz + k) * C)[part] =
        *reinterpret_cast<const uint4 *>(o);
}

// Head and loss: z = bh + sum_c Wh[c] d0[v][c]; with labels, the binary
// cross entropy of sigmoid(z) and its gradient dz = (sigmoid(z) - y) / N.
__global__ void __launch_bounds__(256) k_head(const bf16 *__restrict__ D0, long long V,
                                              const float *__restrict__ Wh,
                                              const float *__restrict__ bh,
                                              const uint8_t *__restrict__ chi, int NX, int NY,
                                              int NZ, int ox, int oy, int oz, int ny, int nz,
                                              float *__restrict__ z_out, float *__restrict__ dz,
                                              double *__restrict__ loss_part)
{
    __shared__ double s_l[8];
    const long long v = (long long)blockIdx.x * 256 + threadIdx.x;
    double l = 0.0;
    if (v < V) {
        float z = *bh;
        const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(D0 + v * 32);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float2 f = __bfloat1622float2(p[c]);
            z = fmaf(Wh[2 * c], f.x, z);
            z = fmaf(Wh[2 * c + 1], f.y, z);
        }
        if (z_out) z_out[v] = z;
        if (chi) {
            const int i = (int)(v / ((long long)ny * nz)), j = (int)((v / nz) % ny),
                      k = (int)(v % nz);
            const float y = chi[((long long)(i + ox) * NY + (j + oy)) * NZ + (k + oz)] ? 1.f : 0.f;
            const double zd = z;
            l = fmax(zd, 0.0) - zd * y + log1p(exp(-fabs(zd)));
            const float sg = 1.f / (1.f + __expf(-z));
            dz[v] = (sg - y) / (float)V;
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) s_l[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0 && loss_part) {
        double s = 0.0;
        for (int q = 0; q < 8; ++q) s += s_l[q];
        loss_part[blockIdx.x] = s;
    }
}

// Head backward: g0[v][c] = Wh[c] dz[v] (FP32); the block's sums of
// d0[v][c] dz[v] (c < 32) and of dz[v] (entry 32) go to part[block][33]
// (summed over blocks in order afterwards into dWh and dbh).
__global__ void __launch_bounds__(256) k_head_bwd(const bf16 *__restrict__ D0, long long V,
                                                  const float *__restrict__ Wh,
                                                  const float *__restrict__ dz,
                                                  float *__restrict__ g0, float *__restrict__ part)
{
    __shared__ float s_w[33][8];
    const long long v = (long long)blockIdx.x * 256 + threadIdx.x;
    float pw[33];
#pragma unroll
    for (int c = 0; c < 33; ++c) pw[c] = 0.f;
    if (v < V) {
        const float d = dz[v];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            g0[v * 32 + c] = Wh[c] * d;
            pw[c] = __bfloat162float(D0[v * 32 + c]) * d;
        }
        pw[32] = d;
    }
#pragma unroll
    for (int c = 0; c < 33; ++c) {
        float s = pw[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) s_w[c][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < 33) {
        float s = 0.f;
        for (int q = 0; q < 8; ++q) s += s_w[threadIdx.x][q];
        part[(long long)blockIdx.x * 33 + threadIdx.x] = s;
    }
}

// dZ = bf16(g * [y > 0]) for a relu layer's output y; the block's sums of
// dZ per channel go to part[block][C] (summed over blocks in order
// afterwards into db).  C divides 256, so thread t only ever sees channel
// t % C: it sums its elements in order, then the threads of a channel are
// added in thread order.
__global__ void __launch_bounds__(256) k_relu_bwd(const float *__restrict__ gsum,
                                                  const bf16 *__restrict__ y, long long V, int C,
                                                  bf16 *__restrict__ dZ, float *__restrict__ part)
{
    __shared__ float s_db[256];
    const long long n = V * C;
    float acc = 0.f;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < n;
         e += (long long)gridDim.x * 256) {
        const float yv = __bfloat162float(y[e]);
        const bf16 d = __float2bfloat16(yv > 0.f ? gsum[e] : 0.f);
        dZ[e] = d;
        acc += __bfloat162float(d);
    }
    s_db[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int k = threadIdx.x; k < 256; k += C) t += s_db[k];
        part[(long long)blockIdx.x * C + threadIdx.x] = t;
    }
}

// From the input gradient dX [v][Ca + Cb] (FP32) of a decoder conv: the
// skip part is added into accA [v][Ca]; the coarse part, summed over the
// 2x2x2 cells that read each coarse cell, is written to gB [u][Cb].
__global__ void k_split_skip(const float *__restrict__ dX, long long V, int Ca, int Cb,
                             float *__restrict__ accA)
{
    const long long n = V * Ca;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long v = e / Ca;
    const int c = (int)(e - v * Ca);
    accA[e] += dX[v * (Ca + Cb) + c];
}

__global__ void k_split_coarse(const float *__restrict__ dX, int nx, int ny, int nz, int Ca,
                               int Cb, float *__restrict__ gB)
{
    const int hx = nx >> 1, hy = ny >> 1, hz = nz >> 1;
    const long long n = (long long)hx * hy * hz * Cb;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long u = e / Cb;
    const int c = (int)(e - u * Cb);
    const int i = (int)(u / ((long long)hy * hz)), j = (int)((u / hz) % hy), k = (int)(u % hz);
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const long long v = ((long long)(2 * i + (d >> 2)) * ny + 2 * j + ((d >> 1) & 1)) * nz +
                            2 * k + (d & 1);
        s += dX[v * (Ca + Cb) + Ca + c];
    }
    gB[e] = s;
}

// acc[v][c] += dP[parent(v)][c] / 8 (gradient through mean pooling).
__global__ void k_pool_bwd(const float *__restrict__ dP, int nx, int ny, int nz, int C,
                           float *__restrict__ acc)
{
    const long long n = (long long)nx * ny * nz * C;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const long long v = e / C;
    const int c = (int)(e - v * C);
    const int i = (int)(v / ((long long)ny * nz)), j = (int)((v / nz) % ny), k = (int)(v % nz);
    const long long u = ((long long)(i >> 1) * (ny >> 1) + (j >> 1)) * (nz >> 1) + (k >> 1);
    acc[e] += 0.125f * dP[u * C + c];
}

// Flat FP32 parameters (per layer W[co][ci][3][3][3] then b) -> bf16
// forward weights Wt[tap][co][cip] and flipped input-gradient weights
// Wd[tap][ci][co] (cip: ci padded; padded entries zero).  fold: the input
// carries each cell's x neighbours as channels dx ci_n + ci (dx = 0, 1, 2
// for x offsets -1, 0, +1), so W[co][ci][dx][b][c] moves to the tap at x
// offset 0, channel dx ci_n + ci, and the other taps are zero.
__global__ void k_pack_weights(const float *__restrict__ W, int co_n, int ci_n, int cip,
                               bool fold, bf16 *__restrict__ Wt, bf16 *__restrict__ Wd)
{
    const long long n = 27ll * co_n * cip;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int tap = (int)(e / ((long long)co_n * cip));
    const int co = (int)((e / cip) % co_n);
    const int ci = (int)(e % cip);
    float w;
    if (fold) {
        const int dx = ci / ci_n, f = ci - dx * ci_n;
        w = tap / 9 == 1 && dx < 3 ? W[((long long)co * ci_n + f) * 27 + dx * 9 + tap % 9] : 0.f;
    } else {
        w = ci < ci_n ? W[((long long)co * ci_n + ci) * 27 + tap] : 0.f;
    }
    const bf16 b = __float2bfloat16(w);
    Wt[e] = b;
    if (Wd) Wd[((long long)(26 - tap) * cip + ci) * co_n + co] = b;
}

// dW[tap][co][cip] (FP32) -> flat gradient order W[co][ci][3][3][3]; with
// fold (the packing above) W[co][ci][dx][b][c] is the x-offset-0 tap (b, c)
// at channel dx ci_n + ci.
__global__ void k_unpack_grad(const float *__restrict__ dW, int co_n, int ci_n, int cip,
                              bool fold, float *__restrict__ g)
{
    const long long n = (long long)co_n * ci_n * 27;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int tap = (int)(e % 27);
    const int ci = (int)((e / 27) % ci_n);
    const int co = (int)(e / (27ll * ci_n));
    g[e] = fold ? dW[((long long)(9 + tap % 9) * co_n + co) * cip + (tap / 9) * ci_n + ci]
                : dW[((long long)tap * co_n + co) * cip + ci];
}

__global__ void k_adam(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ s, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float si = b2 * s[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    s[e] = si;
    th[e] -= lr * (mi / c1) / (sqrtf(si / c2) + eps);
}

__global__ void k_threshold(const float *__restrict__ z, long long V, uint8_t *__restrict__ chi)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V) chi[v] = z[v] > 0.f ? 1 : 0;
}

// Features of a system: asinh((U - C|E|^2) / s), asinh(C|E|^2 / s) and
// the tight-surface labels, as three FP32 planes.
__global__ void k_features(const float *__restrict__ U, const float *__restrict__ Ex,
                           const float *__restrict__ Ey, const float *__restrict__ Ez,
                           const uint8_t *__restrict__ chi_t, float cfa, float inv_s, long long G,
                           float *__restrict__ x)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G) return;
    const float e2 = fmaf(Ex[v], Ex[v], fmaf(Ey[v], Ey[v], Ez[v] * Ez[v]));
    const float c = cfa * e2;
    x[v] = asinhf((U[v] - c) * inv_s);
    x[G + v] = asinhf(c * inv_s);
    x[2 * G + v] = chi_t[v] ? 1.f : 0.f;
}

}  // namespace unet
}  // namespace vesis

// ================================================================ host side
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "vesis.h"

namespace vesis {
namespace unet {

struct Layer {
    int ci_n, cip, co_n, k;
    long long w_off, b_off;     // in the flat parameter vector
    bf16 *Wt = nullptr, *Wd = nullptr;
    bf16 *Wtc = nullptr, *Wdc = nullptr;   // the same in the TMA kernel's layout
    float *dW = nullptr;
};

int tc_tile(int c) { return c % 64 == 0 ? 64 : 32; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of a channels-last activation [nx][ny][nz][C] bf16 with the
// halo box {8 ch, 10 z, 18 y, hx x}; out-of-range cells read as zero.
bool encode_halo_map(CUtensorMap *m, const bf16 *base, int C, int nx, int ny, int nz,
                     int hx = TC_HX)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)nx};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * nz,
                                   (cuuint64_t)C * 2 * nz * ny};
    const cuuint32_t box[4] = {8, (cuuint32_t)TC_HZ, (cuuint32_t)TC_HY, (cuuint32_t)hx};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(base), dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

enum { L_E0, L_E1, L_E2, L_E3, L_D2, L_D1, L_D0, L_HEAD, L_N };

}  // namespace unet
}  // namespace vesis

using namespace vesis;
using namespace vesis::unet;

struct vesis_net_t {
    int dev = 0;
    cudaStream_t st = nullptr;
    int F = 0;
    bool fold = false;            // input layer: x neighbours folded into channels (3 F <= 32)
    long long P = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *s = nullptr;
    Layer L[L_N];
    long long step = 0;
    bool packed = false;
    // activations for the current crop size
    int nx = 0, ny = 0, nz = 0;
    bool train = false;
    bf16 *X0 = nullptr, *e[4] = {}, *p[3] = {}, *d[3] = {};   // d[0] = d0, d[1] = d1, d[2] = d2
    float *z = nullptr, *dz = nullptr;
    double *loss_part = nullptr;
    float *ge[4] = {}, *gd[3] = {}, *dX = nullptr;
    bf16 *dZ = nullptr;
    float *part = nullptr;        // per-block partial gradients, summed in order
    long long part_cap = 0;       // floats
    double *h_loss = nullptr;
    int conv_kind = 1;            // 0 mma.sync, 1 tcgen05 where the shape allows
    bf16 *up = nullptr;           // a decoder's coarse input doubled to its resolution
    long long up_cap = 0;
    int *d_err = nullptr;         // timeout flag of the tcgen05 convolution
    int *h_err = nullptr;
    std::vector<void *> act;      // activation allocations
    std::vector<void *> fixed;    // parameter-sized allocations
};

namespace vesis {
std::string *noalloc_last_error();   // the thread's error message (api.cu)
}

namespace {

std::string *net_err() { return vesis::noalloc_last_error(); }

int nfail(int code, const std::string &msg)
{
    *net_err() = msg;
    return code;
}

#define NCK(x)                                                                     \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) return nfail(VESIS_E_CUDA, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int nalloc(std::vector<void *> &v, T **p, size_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess)
        return nfail(VESIS_E_ALLOC, "device allocation failed");
    v.push_back(q);
    *p = static_cast<T *>(q);
    return VESIS_OK;
}

void free_act(vesis_net n)
{
    for (void *q : n->act) cudaFree(q);
    n->act.clear();
    n->up = nullptr;
    n->up_cap = 0;
    n->nx = n->ny = n->nz = 0;
}

#define NTRY(x)                      \
    do {                             \
        int r_ = (x);                \
        if (r_ != VESIS_OK) return r_; \
    } while (0)

int ensure_act(vesis_net n, int nx, int ny, int nz, bool train)
{
    if (n->nx == nx && n->ny == ny && n->nz == nz && (n->train || !train)) return VESIS_OK;
    NCK(cudaStreamSynchronize(n->st));
    free_act(n);
    const long long V0 = (long long)nx * ny * nz, V1 = V0 / 8, V2 = V1 / 8, V3 = V2 / 8;
    const long long V[4] = {V0, V1, V2, V3};
    auto &A = n->act;
    NTRY(nalloc(A, &n->X0, V0 * kInPad));
    for (int l = 0; l < 4; ++l) NTRY(nalloc(A, &n->e[l], V[l] * kCh[l]));
    for (int l = 0; l < 3; ++l) NTRY(nalloc(A, &n->p[l], V[l + 1] * kCh[l]));
    NTRY(nalloc(A, &n->d[0], V0 * 32));
    NTRY(nalloc(A, &n->d[1], V1 * 32));
    NTRY(nalloc(A, &n->d[2], V2 * 64));
    NTRY(nalloc(A, &n->z, V0));
    NTRY(nalloc(A, &n->up, V0 * 32));    // the largest doubled coarse input (d0's)
    n->up_cap = V0 * 32;
    NTRY(nalloc(A, &n->loss_part, (V0 + 255) / 256));
    if (train) {
        NTRY(nalloc(A, &n->dz, V0));
        for (int l = 0; l < 4; ++l) NTRY(nalloc(A, &n->ge[l], V[l] * kCh[l]));
        NTRY(nalloc(A, &n->gd[0], V0 * 32));
        NTRY(nalloc(A, &n->gd[1], V1 * 32));
        NTRY(nalloc(A, &n->gd[2], V2 * 64));
        long long mx = V0 * 64;
        mx = std::max(mx, V1 * 128);
        mx = std::max(mx, V2 * 256);
        NTRY(nalloc(A, &n->dX, mx));
        NTRY(nalloc(A, &n->dZ, V0 * 32 > V2 * 128 ? V0 * 32 : V2 * 128));
        // partial gradients: the weight gradient's chunks (at most 608 + 27 x
        // 8 x 2 blocks of 64 x 32 entries), the ReLU layers' 608 x 128 and
        // the head's blocks x 33
        long long pc = 16ll << 20;        // at least 16 M floats: the tcgen05 chunks
        pc = std::max(pc, (608ll + 27 * 8 * 2) * 64 * 32);
        pc = std::max(pc, 608ll * 128);
        pc = std::max(pc, (V0 + 255) / 256 * 33);
        NTRY(nalloc(A, &n->part, pc));
        n->part_cap = pc;
    }
    n->nx = nx;
    n->ny = ny;
    n->nz = nz;
    n->train = train;
    return VESIS_OK;
}

unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Launch shape of the row-indexed kernels: rows (i, j) of an nx x ny x nz
// grid on x, per_row items of a row on y in blocks of t threads.
dim3 row_grid(int nx, int ny, long long per_row, int t = 128)
{
    return dim3((unsigned)((long long)nx * ny), (unsigned)((per_row + t - 1) / t));
}

// log2 of the number of 8-channel groups of C channels (C / 8 a power of two).
int log2_groups(int C)
{
    int g = C / 8, s = 0;
    while ((1 << s) < g) ++s;
    return s;
}

// Returns true when the 1x1 head (hw, hb -> hz, a 32-channel layer's
// outputs) was fused into the convolution, whose outputs were then not
// stored; only the TMA kernel fuses it.
bool conv(vesis_net n, int nx, int ny, int nz, const bf16 *A, int Ca, const bf16 *B, int Cb,
          const bf16 *Wt, const bf16 *Wtc, const float *bias, int Cout, void *Y, bool raw,
          int k16 = 2, const float *hw = nullptr, const float *hb = nullptr, float *hz = nullptr,
          bool x1 = false)
{
    ConvArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.V = (long long)nx * ny * nz;
    a.A = A;
    a.Ca = Ca;
    a.B = B;
    a.Cb = Cb;
    a.Wt = Wt;
    a.bias = bias;
    a.Cout = Cout;
    a.Y = Y;
    a.k16 = k16;
    a.x1 = x1;
    count_launch();
    if (n->conv_kind == 1 && ny % TCY == 0 && nz % TCZ == 0 && Ca % 32 == 0 && Cb % 32 == 0 &&
        Cout % 32 == 0) {
        const unsigned bricks = (unsigned)(nx * (ny / TCY) * (nz / TCZ));
        CUtensorMap tm, tmb;
        bool tma_ok = bricks >= 152u * 4u && Wtc &&
                      encode_halo_map(&tm, A, Ca, nx, ny, nz, x1 ? 1 : TC_HX);
        if (tma_ok && Cb > 0) {
            // the coarse input doubled to the output's resolution, so that
            // both inputs arrive by tensor-map boxes
            tma_ok = n->up && (long long)nx * ny * nz * Cb <= n->up_cap &&
                     encode_halo_map(&tmb, n->up, Cb, nx, ny, nz);
            if (tma_ok) {
                count_launch();
                k_upsample<<<row_grid(nx, ny, (long long)nz * (Cb / 8)), 128, 0, n->st>>>(
                    B, nx, ny, nz, Cb, log2_groups(Cb), n->up);
            }
        } else {
            tmb = tm;
        }
        if (tma_ok) {
            // enough bricks for weight-stationary blocks: TMA and bulk copies,
            // nb bricks per block, halved from 512 / NT while that leaves
            // fewer than two blocks per SM
            const int NTt = tc_tile(Cout);
            int bpb = tma_max_nb(NTt);
            while (bpb > 2 && (long long)((bricks + bpb - 1) / bpb) * (Cout / NTt) < 2 * 152) bpb /= 2;
            const unsigned nb = (bricks + bpb - 1) / bpb;
            const bool fuse = hz && !raw && Cout == 32;
            if (fuse) {
                a.hw = hw;
                a.hb = hb;
                a.hz = hz;
            }
            if (tc_tile(Cout) == 64) {
                dim3 tg(nb, Cout / 64);
                if (raw) k_conv_tma<64, true><<<tg, 128, tma_smem_bytes(64), n->st>>>(a, tm, tmb, Wtc, (int)bricks, bpb, n->d_err);
                else k_conv_tma<64, false><<<tg, 128, tma_smem_bytes(64), n->st>>>(a, tm, tmb, Wtc, (int)bricks, bpb, n->d_err);
            } else {
                dim3 tg(nb, Cout / 32);
                if (raw) k_conv_tma<32, true><<<tg, 128, tma_smem_bytes(32), n->st>>>(a, tm, tmb, Wtc, (int)bricks, bpb, n->d_err);
                else k_conv_tma<32, false><<<tg, 128, tma_smem_bytes(32), n->st>>>(a, tm, tmb, Wtc, (int)bricks, bpb, n->d_err);
            }
            return fuse;
        }
        if (Cout % 64 == 0) {
            dim3 tg(bricks, Cout / 64);
            if (raw) k_conv_tc<64, true><<<tg, 128, tc_smem_bytes(64), n->st>>>(a, n->d_err);
            else k_conv_tc<64, false><<<tg, 128, tc_smem_bytes(64), n->st>>>(a, n->d_err);
        } else {
            dim3 tg(bricks, Cout / 32);
            if (raw) k_conv_tc<32, true><<<tg, 128, tc_smem_bytes(32), n->st>>>(a, n->d_err);
            else k_conv_tc<32, false><<<tg, 128, tc_smem_bytes(32), n->st>>>(a, n->d_err);
        }
        return false;
    }
    if (nx % HXB == 0 && ny % HYB == 0 && nz % HZB == 0 && Ca % 32 == 0 && Cb % 32 == 0) {
        const unsigned bricks = (unsigned)((nx / HXB) * (ny / HYB) * (nz / HZB));
        dim3 hg(bricks, Cout / HBN);
        const size_t sm = sizeof(HaloSmem<32>);
        if (raw) k_conv_halo<32, true><<<hg, 128, sm, n->st>>>(a);
        else k_conv_halo<32, false><<<hg, 128, sm, n->st>>>(a);
        return false;
    }
    const int BN = Cout >= 64 ? 64 : 32;
    dim3 grid((unsigned)((a.V + CM - 1) / CM), Cout / BN);
    if (BN == 64) {
        if (raw) k_conv<64, true><<<grid, 128, 0, n->st>>>(a);
        else k_conv<64, false><<<grid, 128, 0, n->st>>>(a);
    } else {
        if (raw) k_conv<32, true><<<grid, 128, 0, n->st>>>(a);
        else k_conv<32, false><<<grid, 128, 0, n->st>>>(a);
    }
    return false;
}

void wgrad(vesis_net n, int nx, int ny, int nz, const bf16 *A, int Ca, const bf16 *B, int Cb,
           const bf16 *dZ, int Cout, float *dW)
{
    // chunk partials in n->part, then one ordered sum into dW
    const int Cin_ = Ca + Cb;
    const long long nw_ = 27ll * Cout * Cin_;
    if (n->conv_kind == 1 && ny % TCY == 0 && nz % TCZ == 0 && Ca % 32 == 0 && Cb % 32 == 0 &&
        Cout % 32 == 0 && (Cout >= Cin_ ? Cin_ : Cout) <= 128) {
        WgradTcArgs t;
        t.nx = nx;
        t.ny = ny;
        t.nz = nz;
        t.A = A;
        t.Ca = Ca;
        t.B = B;
        t.Cb = Cb;
        t.dZ = dZ;
        t.Cout = Cout;
        t.part = n->part;
        t.rows_co = Cout >= Cin_ ? 1 : 0;
        t.N = t.rows_co ? Cin_ : Cout;
        t.taps = std::min(27, 512 / t.N);
        const int groups = (27 + t.taps - 1) / t.taps;
        const int mt = t.rows_co ? 1 : (Cin_ + 127) / 128;
        t.nbricks = nx * (ny / TCY) * (nz / TCZ);
        long long chunks = std::max(1, 152 / (groups * mt));     // one wave
        chunks = std::min<long long>(chunks, t.nbricks);
        chunks = std::min<long long>(chunks, std::max(1ll, n->part_cap / nw_));
        t.bricks_per_chunk = (int)((t.nbricks + chunks - 1) / chunks);
        chunks = (t.nbricks + t.bricks_per_chunk - 1) / t.bricks_per_chunk;
        count_launch(2);
        k_wgrad_tc<<<dim3((unsigned)chunks, (unsigned)groups, (unsigned)mt), 128, WT_SMEM,
                     n->st>>>(t, n->d_err);
        k_sum_parts4<<<nblk(nw_ / 4), 256, 0, n->st>>>(reinterpret_cast<const float4 *>(n->part),
                                                        (int)chunks, nw_ / 4,
                                                        reinterpret_cast<float4 *>(dW));
        return;
    }
    WgradArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.V = (long long)nx * ny * nz;
    a.A = A;
    a.Ca = Ca;
    a.B = B;
    a.Cb = Cb;
    a.dZ = dZ;
    a.Cout = Cout;
    a.part = n->part;
    const int Cin = Ca + Cb;
    const long long tiles = 27ll * (Cin / 32) * ((Cout + 63) / 64);
    // about four blocks per SM in all, in multiples of 32 cells
    long long chunks = std::max(1ll, (152ll * 4) / tiles);
    long long cpb = (a.V + chunks - 1) / chunks;
    cpb = std::max(256ll, (cpb + WK - 1) / WK * WK);
    a.cells_per_block = cpb;
    chunks = (a.V + cpb - 1) / cpb;
    dim3 grid((unsigned)chunks, (unsigned)(27 * (Cin / 32)), (unsigned)((Cout + 63) / 64));
    const long long nw = 27ll * Cout * Cin;
    count_launch(2);
    k_wgrad<<<grid, 128, 0, n->st>>>(a);
    k_sum_parts4<<<nblk(nw / 4), 256, 0, n->st>>>(reinterpret_cast<const float4 *>(n->part),
                                                  (int)chunks, nw / 4,
                                                  reinterpret_cast<float4 *>(dW));
}

// Forward pass of a crop; with labels, the loss partials and dz too.
void forward(vesis_net n, const float *x, int NX, int NY, int NZ, int ox, int oy, int oz,
             const uint8_t *chi)
{
    const int nx = n->nx, ny = n->ny, nz = n->nz;
    const long long V0 = (long long)nx * ny * nz;
    const int r[4][3] = {{nx, ny, nz}, {nx / 2, ny / 2, nz / 2}, {nx / 4, ny / 4, nz / 4},
                         {nx / 8, ny / 8, nz / 8}};
    Layer *L = n->L;
    const float *th = n->theta;
    count_launch();
    if (n->F == 3)
        k_pack_input<3><<<row_grid(nx, ny, nz), 128, 0, n->st>>>(x, n->F, NX, NY, NZ, ox, oy, oz, nx, ny, nz,
                                                     n->fold, n->X0);
    else
        k_pack_input<0><<<row_grid(nx, ny, nz), 128, 0, n->st>>>(x, n->F, NX, NY, NZ, ox, oy, oz, nx, ny, nz,
                                                     n->fold, n->X0);
    conv(n, nx, ny, nz, n->X0, kInPad, nullptr, 0, L[L_E0].Wt, L[L_E0].Wtc, th + L[L_E0].b_off, 32,
         n->e[0], false, ((n->fold ? 3 : 1) * n->F + 15) / 16, nullptr, nullptr, nullptr, n->fold);
    for (int l = 1; l < 4; ++l) {
        count_launch();
        k_pool<<<row_grid(r[l][0], r[l][1], (long long)r[l][2] * (kCh[l - 1] / 8)), 128, 0, n->st>>>(
            n->e[l - 1], r[l - 1][0], r[l - 1][1], r[l - 1][2], kCh[l - 1], log2_groups(kCh[l - 1]),
            n->p[l - 1]);
        conv(n, r[l][0], r[l][1], r[l][2], n->p[l - 1], kCh[l - 1], nullptr, 0, L[l].Wt, L[l].Wtc,
             th + L[l].b_off, kCh[l], n->e[l], false);
    }
    conv(n, r[2][0], r[2][1], r[2][2], n->e[2], 128, n->e[3], 128, L[L_D2].Wt, L[L_D2].Wtc,
         th + L[L_D2].b_off, 64, n->d[2], false);
    conv(n, r[1][0], r[1][1], r[1][2], n->e[1], 64, n->d[2], 64, L[L_D1].Wt, L[L_D1].Wtc,
         th + L[L_D1].b_off, 32, n->d[1], false);
    // without targets (inference) the head may run in d0's epilogue
    const bool fused = conv(n, nx, ny, nz, n->e[0], 32, n->d[1], 32, L[L_D0].Wt, L[L_D0].Wtc,
                            th + L[L_D0].b_off, 32, n->d[0], false, 2, th + L[L_HEAD].w_off,
                            th + L[L_HEAD].b_off, chi ? nullptr : n->z);
    if (fused) return;
    count_launch();
    k_head<<<nblk(V0), 256, 0, n->st>>>(n->d[0], V0, th + L[L_HEAD].w_off,
                                        th + L[L_HEAD].b_off, chi, NX, NY, NZ, ox, oy, oz, ny, nz, n->z,
                                        chi ? n->dz : nullptr, chi ? n->loss_part : nullptr);
}

int pack_weights(vesis_net n)
{
    for (int l = 0; l < L_HEAD; ++l) {
        Layer &y = n->L[l];
        count_launch();
        k_pack_weights<<<nblk(27ll * y.co_n * y.cip), 256, 0, n->st>>>(
            n->theta + y.w_off, y.co_n, y.ci_n, y.cip, l == L_E0 && n->fold, y.Wt, y.Wd);
        count_launch(2);
        k_pack_tc<<<nblk(27ll * y.co_n * y.cip), 256, 0, n->st>>>(y.Wt, y.co_n, y.cip,
                                                                 tc_tile(y.co_n), y.Wtc);
        k_pack_tc<<<nblk(27ll * y.co_n * y.cip), 256, 0, n->st>>>(y.Wd, y.cip, y.co_n,
                                                                 tc_tile(y.cip), y.Wdc);
    }
    n->packed = true;
    return VESIS_OK;
}

}  // namespace

extern "C" {

int vesis_net_create(int n_features, void *cuda_stream, vesis_net *out)
{
    if (!out) return nfail(VESIS_E_ARG, "out is NULL");
    *out = nullptr;
    if (n_features < 1 || n_features > kInPad)
        return nfail(VESIS_E_ARG, "n_features must be in 1..32");
    vesis_net n = new vesis_net_t();
    n->st = (cudaStream_t)cuda_stream;
    n->F = n_features;
    n->fold = 3 * n_features <= kInPad;
    if (cudaGetDevice(&n->dev) != cudaSuccess) {
        delete n;
        return nfail(VESIS_E_CUDA, "no CUDA device");
    }
    const int ci[L_N] = {n_features, 32, 64, 128, 256, 128, 64, 32};
    const int cip[L_N] = {kInPad, 32, 64, 128, 256, 128, 64, 32};
    const int co[L_N] = {32, 64, 128, 128, 64, 32, 32, 1};
    long long o = 0;
    for (int l = 0; l < L_N; ++l) {
        Layer &y = n->L[l];
        y.ci_n = ci[l];
        y.cip = cip[l];
        y.co_n = co[l];
        y.k = l == L_HEAD ? 1 : 3;
        y.w_off = o;
        o += (long long)co[l] * ci[l] * y.k * y.k * y.k;
        y.b_off = o;
        o += co[l];
    }
    n->P = o;
    int rc = VESIS_OK;
    auto &A = n->fixed;
    if (rc == VESIS_OK) rc = nalloc(A, &n->theta, o);
    if (rc == VESIS_OK) rc = nalloc(A, &n->grad, o);
    if (rc == VESIS_OK) rc = nalloc(A, &n->m, o);
    if (rc == VESIS_OK) rc = nalloc(A, &n->s, o);
    for (int l = 0; l < L_HEAD && rc == VESIS_OK; ++l) {
        Layer &y = n->L[l];
        const long long nw = 27ll * y.co_n * y.cip;
        rc = nalloc(A, &y.Wt, nw);
        if (rc == VESIS_OK) rc = nalloc(A, &y.Wd, nw);
        if (rc == VESIS_OK) rc = nalloc(A, &y.Wtc, nw);
        if (rc == VESIS_OK) rc = nalloc(A, &y.Wdc, nw);
        if (rc == VESIS_OK) rc = nalloc(A, &y.dW, nw);
    }
    if (rc == VESIS_OK &&
        (cudaFuncSetAttribute(k_conv_halo<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(HaloSmem<32>)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_halo<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(HaloSmem<32>)) != cudaSuccess))
        rc = nfail(VESIS_E_CUDA, "shared memory attribute of the conv kernel");
    if (rc == VESIS_OK &&
        (cudaFuncSetAttribute(k_conv_tc<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc_smem_bytes(32)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tc<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc_smem_bytes(32)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tc<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc_smem_bytes(64)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tc<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tc_smem_bytes(64)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tma<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tma_smem_bytes(32)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tma<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tma_smem_bytes(32)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tma<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tma_smem_bytes(64)) != cudaSuccess ||
         cudaFuncSetAttribute(k_conv_tma<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              tma_smem_bytes(64)) != cudaSuccess ||
         cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              WT_SMEM) != cudaSuccess))
        rc = nfail(VESIS_E_CUDA, "shared memory attribute of the tensor-core conv kernel");
    if (rc == VESIS_OK) rc = nalloc(A, &n->d_err, 1);
    if (rc == VESIS_OK && cudaMallocHost(&n->h_err, sizeof(int)) != cudaSuccess)
        rc = nfail(VESIS_E_ALLOC, "pinned allocation failed");
    if (rc == VESIS_OK) cudaMemsetAsync(n->d_err, 0, sizeof(int), n->st);
    if (rc == VESIS_OK && cudaMallocHost(&n->h_loss, sizeof(double)) != cudaSuccess)
        rc = nfail(VESIS_E_ALLOC, "pinned allocation failed");
    if (rc == VESIS_OK) {
        cudaMemsetAsync(n->theta, 0, o * sizeof(float), n->st);
        cudaMemsetAsync(n->m, 0, o * sizeof(float), n->st);
        cudaMemsetAsync(n->s, 0, o * sizeof(float), n->st);
        if (cudaStreamSynchronize(n->st) != cudaSuccess)
            rc = nfail(VESIS_E_CUDA, "stream synchronisation failed");
    }
    if (rc != VESIS_OK) {
        std::string keep = *net_err();
        vesis_net_destroy(n);
        *net_err() = keep;
        return rc;
    }
    *out = n;
    return VESIS_OK;
}

int vesis_net_param_count(vesis_net n, long long *count)
{
    if (!n || !count) return nfail(VESIS_E_ARG, "NULL argument");
    *count = n->P;
    return VESIS_OK;
}

int vesis_net_set_params(vesis_net n, const float *theta)
{
    if (!n || !theta) return nfail(VESIS_E_ARG, "NULL argument");
    for (long long i = 0; i < n->P; ++i)
        if (!std::isfinite(theta[i])) return nfail(VESIS_E_NAN, "non-finite parameter");
    NCK(cudaMemcpyAsync(n->theta, theta, n->P * sizeof(float), cudaMemcpyHostToDevice, n->st));
    NCK(cudaMemsetAsync(n->m, 0, n->P * sizeof(float), n->st));
    NCK(cudaMemsetAsync(n->s, 0, n->P * sizeof(float), n->st));
    NCK(cudaStreamSynchronize(n->st));
    n->step = 0;
    n->packed = false;
    return VESIS_OK;
}

int vesis_net_get_params(vesis_net n, float *theta)
{
    if (!n || !theta) return nfail(VESIS_E_ARG, "NULL argument");
    NCK(cudaMemcpyAsync(theta, n->theta, n->P * sizeof(float), cudaMemcpyDeviceToHost, n->st));
    NCK(cudaStreamSynchronize(n->st));
    return VESIS_OK;
}

static int check_crop(int NX, int NY, int NZ, const int *crop, int c[6])
{
    if (NX < 1 || NY < 1 || NZ < 1) return nfail(VESIS_E_ARG, "bad grid dimensions");
    if (crop) {
        for (int i = 0; i < 6; ++i) c[i] = crop[i];
    } else {
        c[0] = c[1] = c[2] = 0;
        c[3] = NX;
        c[4] = NY;
        c[5] = NZ;
    }
    const int N[3] = {NX, NY, NZ};
    for (int d = 0; d < 3; ++d) {
        if (c[3 + d] < 8 || c[3 + d] % 8 != 0)
            return nfail(VESIS_E_ARG, "crop dimensions must be positive multiples of 8");
        if (c[d] < 0 || c[d] + c[3 + d] > N[d]) return nfail(VESIS_E_ARG, "crop outside the grid");
    }
    if ((long long)c[3] * c[4] * c[5] > 2147483647ll)
        return nfail(VESIS_E_ARG, "crop has more than 2^31-1 cells");
    return VESIS_OK;
}

int vesis_net_forward(vesis_net n, const float *x_dev, int NX, int NY, int NZ, const int *crop,
                      float *logit_dev, uint8_t *chi_dev)
{
    if (!n || !x_dev) return nfail(VESIS_E_ARG, "NULL argument");
    int c[6];
    NTRY(check_crop(NX, NY, NZ, crop, c));
    NTRY(ensure_act(n, c[3], c[4], c[5], false));
    if (!n->packed) pack_weights(n);
    forward(n, x_dev, NX, NY, NZ, c[0], c[1], c[2], nullptr);
    const long long V = (long long)c[3] * c[4] * c[5];
    if (logit_dev)
        NCK(cudaMemcpyAsync(logit_dev, n->z, V * sizeof(float), cudaMemcpyDeviceToDevice, n->st));
    if (chi_dev) {
        count_launch();
        k_threshold<<<nblk(V), 256, 0, n->st>>>(n->z, V, chi_dev);
    }
    NCK(cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->st));
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(n->st));
    if (*n->h_err) return nfail(VESIS_E_CUDA, "tensor-core convolution: mbarrier wait timed out");
    return VESIS_OK;
}

int vesis_net_set_conv_kernel(vesis_net n, int kind)
{
    if (!n) return nfail(VESIS_E_ARG, "NULL net");
    if (kind != 0 && kind != 1) return nfail(VESIS_E_ARG, "kind must be 0 or 1");
    n->conv_kind = kind;
    return VESIS_OK;
}

int vesis_net_loss_grad(vesis_net n, const float *x_dev, const uint8_t *chi_dev, int NX, int NY,
                        int NZ, const int *crop, double *loss_out, float *grad_host)
{
    if (!n || !x_dev || !chi_dev) return nfail(VESIS_E_ARG, "NULL argument");
    int c[6];
    NTRY(check_crop(NX, NY, NZ, crop, c));
    NTRY(ensure_act(n, c[3], c[4], c[5], true));
    if (!n->packed) pack_weights(n);
    const int nx = c[3], ny = c[4], nz = c[5];
    const int r[4][3] = {{nx, ny, nz}, {nx / 2, ny / 2, nz / 2}, {nx / 4, ny / 4, nz / 4},
                         {nx / 8, ny / 8, nz / 8}};
    long long V[4];
    for (int l = 0; l < 4; ++l) V[l] = (long long)r[l][0] * r[l][1] * r[l][2];
    forward(n, x_dev, NX, NY, NZ, c[0], c[1], c[2], chi_dev);
    cudaStream_t st = n->st;
    Layer *L = n->L;
    NCK(cudaMemsetAsync(n->grad, 0, n->P * sizeof(float), st));
    for (int l = 0; l < L_HEAD; ++l)
        NCK(cudaMemsetAsync(L[l].dW, 0, 27ll * L[l].co_n * L[l].cip * sizeof(float), st));
    for (int l = 0; l < 3; ++l)      // e3's gradient is written whole
        NCK(cudaMemsetAsync(n->ge[l], 0, V[l] * kCh[l] * sizeof(float), st));
    // head
    count_launch();
    k_head_bwd<<<nblk(V[0]), 256, 0, st>>>(n->d[0], V[0], n->theta + L[L_HEAD].w_off, n->dz,
                                           n->gd[0], n->part);
    count_launch();
    k_sum_parts_tree<<<33, 256, 0, st>>>(n->part, (int)nblk(V[0]), 33, n->grad + L[L_HEAD].w_off);
    auto relu_bwd = [&](const float *g, const bf16 *y, long long Vl, int C, float *db) {
        count_launch(2);
        const long long nb = std::min<long long>(nblk(Vl * C), 4 * 152);
        k_relu_bwd<<<(unsigned)nb, 256, 0, st>>>(g, y, Vl, C, n->dZ, n->part);
        k_sum_parts_tree<<<C, 256, 0, st>>>(n->part, (int)nb, C, db);
    };
    auto unpack = [&](int l) {
        Layer &y = L[l];
        count_launch();
        k_unpack_grad<<<nblk(27ll * y.co_n * y.ci_n), 256, 0, st>>>(
            y.dW, y.co_n, y.ci_n, y.cip, l == L_E0 && n->fold, n->grad + y.w_off);
    };
    // decoder: d0 (R0), d1 (R1), d2 (R2); skip inputs e0, e1, e2; coarse d1, d2, e3
    struct Dec {
        int l, lev, Ca, Cb, Cout;
        bf16 *skip, *coarse, *out;
        float *gskip, *gout, *gcoarse;
    } dec[3] = {
        {L_D0, 0, 32, 32, 32, n->e[0], n->d[1], n->d[0], n->ge[0], n->gd[0], n->gd[1]},
        {L_D1, 1, 64, 64, 32, n->e[1], n->d[2], n->d[1], n->ge[1], n->gd[1], n->gd[2]},
        {L_D2, 2, 128, 128, 64, n->e[2], n->e[3], n->d[2], n->ge[2], n->gd[2], n->ge[3]},
    };
    for (auto &D : dec) {
        const int *R = r[D.lev];
        const long long Vl = V[D.lev];
        relu_bwd(D.gout, D.out, Vl, D.Cout, n->grad + L[D.l].b_off);
        wgrad(n, R[0], R[1], R[2], D.skip, D.Ca, D.coarse, D.Cb, n->dZ, D.Cout, L[D.l].dW);
        unpack(D.l);
        conv(n, R[0], R[1], R[2], n->dZ, D.Cout, nullptr, 0, L[D.l].Wd, L[D.l].Wdc, nullptr,
             D.Ca + D.Cb, n->dX, true);
        count_launch(2);
        k_split_skip<<<nblk(Vl * D.Ca), 256, 0, st>>>(n->dX, Vl, D.Ca, D.Cb, D.gskip);
        k_split_coarse<<<nblk(V[D.lev + 1] * D.Cb), 256, 0, st>>>(n->dX, R[0], R[1], R[2], D.Ca,
                                                                 D.Cb, D.gcoarse);
    }
    // encoder: e3 (R3, input p2), e2 (R2, input p1), e1 (R1, input p0), e0 (R0, input X0)
    for (int l = 3; l >= 0; --l) {
        const int *R = r[l];
        const long long Vl = V[l];
        const bf16 *in = l == 0 ? n->X0 : n->p[l - 1];
        const int Cin = l == 0 ? kInPad : kCh[l - 1];
        relu_bwd(n->ge[l], n->e[l], Vl, kCh[l], n->grad + L[l].b_off);
        wgrad(n, R[0], R[1], R[2], in, Cin, nullptr, 0, n->dZ, kCh[l], L[l].dW);
        unpack(l);
        if (l > 0) {
            conv(n, R[0], R[1], R[2], n->dZ, kCh[l], nullptr, 0, L[l].Wd, L[l].Wdc, nullptr, Cin,
                 n->dX, true);
            count_launch();
            k_pool_bwd<<<nblk(V[l - 1] * Cin), 256, 0, st>>>(n->dX, r[l - 1][0], r[l - 1][1],
                                                             r[l - 1][2], Cin, n->ge[l - 1]);
        }
    }
    launch_sum_doubles(n->loss_part, (int)nblk(V[0]), reinterpret_cast<double *>(n->dz), 0, st);
    NCK(cudaMemcpyAsync(n->h_loss, n->dz, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_host)
        NCK(cudaMemcpyAsync(grad_host, n->grad, n->P * sizeof(float), cudaMemcpyDeviceToHost, st));
    NCK(cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(st));
    if (*n->h_err) return nfail(VESIS_E_CUDA, "tensor-core convolution: mbarrier wait timed out");
    if (loss_out) *loss_out = *n->h_loss / (double)V[0];
    if (!std::isfinite(*n->h_loss)) return nfail(VESIS_E_NAN, "non-finite loss");
    return VESIS_OK;
}

int vesis_net_adam_step(vesis_net n, double lr, double beta1, double beta2, double eps)
{
    if (!n) return nfail(VESIS_E_ARG, "NULL net");
    if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) ||
        !(eps > 0.0))
        return nfail(VESIS_E_ARG, "invalid Adam constants");
    ++n->step;
    const double c1 = 1.0 - std::pow(beta1, (double)n->step);
    const double c2 = 1.0 - std::pow(beta2, (double)n->step);
    count_launch();
    k_adam<<<nblk(n->P), 256, 0, n->st>>>(n->theta, n->grad, n->m, n->s, n->P, (float)lr,
                                          (float)beta1, (float)beta2, (float)eps, (float)c1,
                                          (float)c2);
    NCK(cudaGetLastError());
    n->packed = false;
    return VESIS_OK;
}

int vesis_net_destroy(vesis_net n)
{
    if (!n) return VESIS_OK;
    cudaStreamSynchronize(n->st);
    free_act(n);
    for (void *q : n->fixed) cudaFree(q);
    if (n->h_loss) cudaFreeHost(n->h_loss);
    if (n->h_err) cudaFreeHost(n->h_err);
    delete n;
    return VESIS_OK;
}

}  // extern "C"

namespace vesis {
void launch_features(const float *U, const float *E, long long G, const uint8_t *chi_t,
                     float cfa, float scale, float *x, cudaStream_t st)
{
    count_launch();
    unet::k_features<<<(unsigned)((G + 255) / 256), 256, 0, st>>>(
        U, E, E + G, E + 2 * G, chi_t, cfa, 1.f / scale, G, x);
}
}  // namespace vesis
