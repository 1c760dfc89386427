// Anchor -> neural Gaussian decoder (Sec. III-A, Eq. 1-5) and its backward.
//
// Forward, one block per 128 anchors (block order from an atomic ticket):
//   1. cull the anchor (camera depth, projected centre inside the widened image)
//   2. Eq. 3: delta = |x^a - x^c|, d = (x^a - x^c) / delta
//   3. Eq. 2: [f, d, delta] through three LINEAR-ReLU-LINEAR MLPs, either
//      FP32 FMA (one thread per anchor, weights in shared memory) or BF16
//      tensor cores (mma.sync m16n8k16, FP32 accumulation; each warp runs two
//      16-anchor tiles: 36->96 hidden, then 32->{10,30,70} per MLP)
//   4. heads: tanh opacity (valid iff > 0), sigmoid colour (Eq. 4), sigmoid
//      scale times the anchor scaling (Eq. 5), normalised quaternion
//   5. Eq. 1 positions, and compaction in (anchor, m) order: per-anchor valid
//      counts are scanned inside the block and offset by a decoupled look-back
//      over earlier blocks, so the decode writes compacted output directly.
// Backward, one block per 128 anchors: recompute the activations, back-propagate
// through heads and MLPs per anchor, then reduce the weight gradients over the
// block's anchors in shared memory (one atomic per parameter per block).
#include <cuda_bf16.h>

#include <type_traits>

#include "internal.h"
#include "prims.cuh"
#include "profiler.h"

namespace vpgs {

#ifndef VPGS_DECODE_BWD_MMA
#define VPGS_DECODE_BWD_MMA 1  // BF16 form: backward on tensor cores (0: the FP32-FMA kernel)
#endif

constexpr int kDecAnchors = 64;    // anchors per forward block
constexpr int kDecThreads = 128;   // threads per forward block (two per anchor)
constexpr int kFeat = 32, kIn = 36, kHid = 32, kMaxK = 10;
constexpr int kOutStride = 121;    // per-anchor row of layer-2 outputs in shared memory
constexpr int kColOpa = 0, kColCol = 16, kColCov = 48;  // column bases (padded to n8 tiles)
constexpr int kInPad = 56;         // bf16 row stride of the staged inputs / W1 rows
constexpr int kW2Pad = 40;         // bf16 row stride of W2 rows

struct DecParams {
    const float *anchors, *scaling, *offsets;
    const void *features;
    int64_t A;
    int K;
    int feat_bf16;
    const float *params;
    int bf16;
    float fx, fy, cx, cy;
    int W, H;
    float near_z, guard;
};

// flat parameter offsets of MLP j (opacity, colour, covariance)
struct MlpOff {
    int w1, b1, w2, b2, out;
};

VPGS_HD MlpOff mlp_off(int K, int j) {
    const int outs[3] = {K, 3 * K, 7 * K};
    int o = 0;
    for (int q = 0; q < j; ++q) o += kIn * kHid + kHid + outs[q] * kHid + outs[q];
    MlpOff m;
    m.w1 = o;
    m.b1 = o + kIn * kHid;
    m.w2 = m.b1 + kHid;
    m.b2 = m.w2 + outs[j] * kHid;
    m.out = outs[j];
    return m;
}

VPGS_HD int n_params(int K) {
    MlpOff m = mlp_off(K, 2);
    return m.b2 + m.out;
}

VPGS_D float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

VPGS_D float sigmoidf_(float x) { return 1.0f / (1.0f + expf(-x)); }

// camera data shared by the block
struct DecCam {
    float R[9], t[3], xc[3];
};

VPGS_D void load_dec_cam(const double *T, DecCam &c) {
    double Rd[9], td[3];
    for (int k = 0; k < 9; ++k) Rd[k] = T[4 * (k / 3) + (k % 3)];
    for (int r = 0; r < 3; ++r) td[r] = T[4 * r + 3];
    for (int k = 0; k < 9; ++k) c.R[k] = (float)Rd[k];
    for (int r = 0; r < 3; ++r) {
        c.t[r] = (float)td[r];
        c.xc[r] = (float)(-(Rd[r] * td[0] + Rd[3 + r] * td[1] + Rd[6 + r] * td[2]));
    }
}

// per-anchor inputs: cull decision and the 36 network inputs (f, d, delta)
VPGS_D bool anchor_inputs(const DecParams &p, const DecCam &c, int64_t a, float in[kIn]) {
    const float x = p.anchors[3 * a], y = p.anchors[3 * a + 1], z = p.anchors[3 * a + 2];
    const float pz = c.R[6] * x + c.R[7] * y + c.R[8] * z + c.t[2];
    const float px = c.R[0] * x + c.R[1] * y + c.R[2] * z + c.t[0];
    const float py = c.R[3] * x + c.R[4] * y + c.R[5] * z + c.t[1];
    bool keep = pz > p.near_z;
    if (keep) {
        const float u = p.fx * px / pz + p.cx, v = p.fy * py / pz + p.cy;
        keep = u >= -p.guard * p.W && u <= (1.f + p.guard) * p.W && v >= -p.guard * p.H &&
               v <= (1.f + p.guard) * p.H;
    }
    if (p.feat_bf16) {
        const __nv_bfloat16 *f = reinterpret_cast<const __nv_bfloat16 *>(p.features) + kFeat * a;
        for (int k = 0; k < kFeat; ++k) in[k] = __bfloat162float(f[k]);
    } else {
        const float4 *f = reinterpret_cast<const float4 *>(static_cast<const float *>(p.features) + kFeat * a);
        for (int k = 0; k < kFeat / 4; ++k) {
            const float4 q = f[k];
            in[4 * k] = q.x; in[4 * k + 1] = q.y; in[4 * k + 2] = q.z; in[4 * k + 3] = q.w;
        }
    }
    const float dx = x - c.xc[0], dy = y - c.xc[1], dz = z - c.xc[2];
    const float dl = sqrtf(dx * dx + dy * dy + dz * dz);
    in[32] = dx / dl;
    in[33] = dy / dl;
    in[34] = dz / dl;
    in[35] = dl;
    if (p.bf16)
        for (int k = 0; k < kIn; ++k) in[k] = bf16r(in[k]);
    return keep;
}

VPGS_D void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                           uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

VPGS_D uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

struct DecOut {
    float *means, *scales, *quats, *opac, *colors;
    int32_t *n_out, *src_index;
};

// dynamic shared memory of the forward kernel
// The forward's weights in the layout its blocks use: BF16 W1 rows [3 x 32]
// [kInPad], BF16 W2 rows [120][kW2Pad] (outputs padded per MLP), FP32 biases.
// Prepared once per call by decode_weights_kernel (the FP32 form keeps the
// flat FP32 parameters in the same region) and copied into each block's
// shared memory as 16-byte words.
struct DecWts {
    __nv_bfloat16 w1[96 * kInPad];
    __nv_bfloat16 w2[120 * kW2Pad];
    float b1[96];
    float b2[120];
};
constexpr int kDecWtsBytes = 48 * 1024;  // room for the forward's forms and the backward's layouts
static_assert(sizeof(DecWts) % 16 == 0 && sizeof(DecWts) <= kDecWtsBytes, "prepared weights: 16-byte words");

struct DecFwdSmem {
    float out[kDecAnchors * kOutStride];
    union {
        float w[8192];  // FP32 weights (n_params(10) = 7182)
        struct {
            DecWts wt;
            __nv_bfloat16 in[kDecAnchors * kInPad];
        } h;
    } u;
    uint16_t slot[kDecAnchors * kMaxK];  // per output slot of the block: local anchor << 4 | m
    float mean[kDecAnchors * 3 * kMaxK]; // per anchor: the means of its Gaussians
};

__global__ void __launch_bounds__(256) decode_weights_kernel(DecParams p, DecWts *wts) {
    grid_dep_enter();
    const int K = p.K, tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (!p.bf16) {
        float *w = reinterpret_cast<float *>(wts);
        for (int i = tid; i < n_params(K); i += stride) w[i] = p.params[i];
        return;
    }
    for (int i = tid; i < 96 * kInPad; i += stride) {
        const int r = i / kInPad, c = i % kInPad;
        const MlpOff m = mlp_off(K, r / 32);
        wts->w1[i] = __float2bfloat16_rn(c < kIn ? p.params[m.w1 + (r % 32) * kIn + c] : 0.f);
    }
    for (int i = tid; i < 120 * kW2Pad; i += stride) {
        const int r = i / kW2Pad, c = i % kW2Pad;
        const int j = r < kColCol ? 0 : (r < kColCov ? 1 : 2);
        const int base = j == 0 ? kColOpa : (j == 1 ? kColCol : kColCov);
        const MlpOff m = mlp_off(K, j);
        const int n = r - base;
        wts->w2[i] = __float2bfloat16_rn((c < kHid && n < m.out) ? p.params[m.w2 + n * kHid + c] : 0.f);
    }
    for (int i = tid; i < 96; i += stride) wts->b1[i] = p.params[mlp_off(K, i / 32).b1 + i % 32];
    for (int i = tid; i < 120; i += stride) {
        const int j = i < kColCol ? 0 : (i < kColCov ? 1 : 2);
        const int base = j == 0 ? kColOpa : (j == 1 ? kColCol : kColCov);
        const MlpOff m = mlp_off(K, j);
        wts->b2[i] = (i - base < m.out) ? p.params[m.b2 + i - base] : 0.f;
    }
}

// FP32 form: MLP j of one anchor, outputs into its row
VPGS_D void mlp_fp32(const float *w, int K, int j, const float (&in)[kIn], float *orow) {
    const MlpOff m = mlp_off(K, j);
    float h[kHid];
#pragma unroll
    for (int q = 0; q < kHid; ++q) {
        const float *wr = w + m.w1 + q * kIn;
        float acc = w[m.b1 + q];
#pragma unroll
        for (int k = 0; k < kIn; ++k) acc = fmaf(wr[k], in[k], acc);
        h[q] = fmaxf(acc, 0.f);
    }
    const int base = j == 0 ? kColOpa : (j == 1 ? kColCol : kColCov);
    for (int n = 0; n < m.out; ++n) {
        const float *wr = w + m.w2 + n * kHid;
        float acc = w[m.b2 + n];
#pragma unroll
        for (int k = 0; k < kHid; ++k) acc = fmaf(wr[k], h[k], acc);
        orow[base + n] = acc;
    }
}

// Resident blocks of kDecThreads threads each load the prepared weights once,
// then decode chunks of kDecAnchors anchors taken from a ticket: thread t < 64 owns
// anchor t for its inputs and its valid-Gaussian count; in the FP32 form
// threads t and t + 64 split its three MLPs (0 and 1 / 2: nearly equal
// work); in the BF16 form each warp runs one 16-anchor tile on tensor cores,
// the opacity head before the others so that the block's count is published
// early.  The head outputs become the Gaussians' values in shared memory while
// the block's compaction offset is resolved; then the outputs are copied one
// Gaussian per thread in output order, so consecutive threads write
// consecutive entries.
__global__ void __launch_bounds__(kDecThreads)
decode_fwd_kernel(DecParams p, const double *__restrict__ T, DecOut o, const DecWts *__restrict__ wts,
                  uint32_t *ticket, unsigned long long *look, uint32_t *status) {
    grid_dep_enter();
    extern __shared__ __align__(16) unsigned char dsm[];
    DecFwdSmem &S = *reinterpret_cast<DecFwdSmem *>(dsm);
    __shared__ uint32_t s_bid, s_base, s_total;
    __shared__ uint32_t s_wsum[kDecThreads / 32];
    __shared__ DecCam s_cam;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) load_dec_cam(T, s_cam);
    const int K = p.K;
    {
        // the prepared weights into shared memory once per block, 16-byte words
        // (both forms start at the union's first byte)
        const int words = p.bf16 ? (int)(sizeof(DecWts) / 16) : (n_params(K) + 3) / 4;
        const uint4 *src = reinterpret_cast<const uint4 *>(wts);
        uint4 *dst = reinterpret_cast<uint4 *>(&S.u);
        for (int i = tid; i < words; i += kDecThreads) dst[i] = src[i];
    }
    // chunks of kDecAnchors anchors in ticket order (the look-back only waits on
    // chunks handed out earlier, each held by a running block)
    for (;;) {
    if (tid == 0) s_bid = atomicAdd(ticket, 1u);
    __syncthreads();  // also: the previous chunk's shared reads are done
    const int64_t bid = s_bid;
    if (bid * kDecAnchors >= p.A) return;
    const int la = tid & (kDecAnchors - 1);  // the block-local anchor this thread reads
    const int64_t a = bid * kDecAnchors + la;
    const bool live = a < p.A;
    float in[kIn];
    bool keep = false;
    if (live && (!p.bf16 || tid < kDecAnchors)) keep = anchor_inputs(p, s_cam, a, in);
    float *orow = S.out + la * kOutStride;
    const int g = lane >> 2, t4 = lane & 3;
    const int r0 = warp * 16;
    float acc[12][4];  // BF16 form: layer 1 of the three MLPs for rows r0 .. r0 + 15
    if (p.bf16) {
        // stage the (already BF16-rounded) inputs, then tensor-core tiles
        if (tid < kDecAnchors) {
            __nv_bfloat16 *irow = S.u.h.in + tid * kInPad;
            for (int k = 0; k < kInPad; ++k) irow[k] = __float2bfloat16_rn(live && k < kIn ? in[k] : 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int nt = 0; nt < 12; ++nt) {
            const float b0 = S.u.h.wt.b1[8 * nt + 2 * t4], b1v = S.u.h.wt.b1[8 * nt + 2 * t4 + 1];
            acc[nt][0] = b0; acc[nt][1] = b1v; acc[nt][2] = b0; acc[nt][3] = b1v;
        }
        const __nv_bfloat16 *A0 = S.u.h.in + (r0 + g) * kInPad, *A1 = S.u.h.in + (r0 + g + 8) * kInPad;
#pragma unroll
        for (int ks = 0; ks < 3; ++ks) {
            const int c0 = 16 * ks + 2 * t4;
            const uint32_t a0 = *reinterpret_cast<const uint32_t *>(A0 + c0);
            const uint32_t a1 = *reinterpret_cast<const uint32_t *>(A1 + c0);
            const uint32_t a2 = *reinterpret_cast<const uint32_t *>(A0 + c0 + 8);
            const uint32_t a3 = *reinterpret_cast<const uint32_t *>(A1 + c0 + 8);
#pragma unroll
            for (int nt = 0; nt < 12; ++nt) {
                const __nv_bfloat16 *Brow = S.u.h.wt.w1 + (8 * nt + g) * kInPad;
                mma_bf16_16816(acc[nt], a0, a1, a2, a3, *reinterpret_cast<const uint32_t *>(Brow + c0),
                               *reinterpret_cast<const uint32_t *>(Brow + c0 + 8));
            }
        }
    }
    // head of MLP j into the anchors' rows (BF16 form: layer 2 on tensor cores,
    // the hidden layer (ReLU, BF16) straight from the accumulators)
    auto head = [&](auto J) {
        constexpr int j = decltype(J)::value;
        constexpr int ntiles = j == 0 ? 2 : (j == 1 ? 4 : 9);
        constexpr int base = j == 0 ? kColOpa : (j == 1 ? kColCol : kColCov);
        uint32_t ha[2][4];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const float *x0 = acc[4 * j + 2 * kk], *x1 = acc[4 * j + 2 * kk + 1];
            ha[kk][0] = pack_bf16(fmaxf(x0[0], 0.f), fmaxf(x0[1], 0.f));
            ha[kk][1] = pack_bf16(fmaxf(x0[2], 0.f), fmaxf(x0[3], 0.f));
            ha[kk][2] = pack_bf16(fmaxf(x1[0], 0.f), fmaxf(x1[1], 0.f));
            ha[kk][3] = pack_bf16(fmaxf(x1[2], 0.f), fmaxf(x1[3], 0.f));
        }
        for (int nt = 0; nt < ntiles; ++nt) {
            const int col = base + 8 * nt + 2 * t4;
            float d[4] = {S.u.h.wt.b2[col], S.u.h.wt.b2[col + 1], S.u.h.wt.b2[col], S.u.h.wt.b2[col + 1]};
            const __nv_bfloat16 *Brow = S.u.h.wt.w2 + (base + 8 * nt + g) * kW2Pad;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const int c0 = 16 * kk + 2 * t4;
                mma_bf16_16816(d, ha[kk][0], ha[kk][1], ha[kk][2], ha[kk][3],
                               *reinterpret_cast<const uint32_t *>(Brow + c0),
                               *reinterpret_cast<const uint32_t *>(Brow + c0 + 8));
            }
            float *o0 = S.out + (r0 + g) * kOutStride + col;
            float *o1 = S.out + (r0 + g + 8) * kOutStride + col;
            o0[0] = d[0]; o0[1] = d[1]; o1[0] = d[2]; o1[1] = d[3];
        }
    };
    // BF16 form: the opacity head first (its outputs decide which Gaussians
    // survive), so the block publishes its count before the colour and covariance
    // heads.  FP32 form: threads t and t + 64 split the three MLPs of anchor t
    // (0 and 1 / 2: nearly equal work), all before the count
    if (!p.bf16) {
        if (keep) {
            if (tid < kDecAnchors) {
                mlp_fp32(S.u.w, K, 0, in, orow);
                mlp_fp32(S.u.w, K, 1, in, orow);
            } else {
                mlp_fp32(S.u.w, K, 2, in, orow);
            }
        }
    } else {
        head(std::integral_constant<int, 0>{});
    }
    __syncthreads();
    // valid Gaussians of each anchor (threads < kDecAnchors), their block-local starts
    uint32_t mask = 0;
    if (tid < kDecAnchors && keep)
        for (int m = 0; m < K; ++m)
            if (orow[kColOpa + m] > 0.f) mask |= 1u << m;
    const uint32_t cnt = __popc(mask);
    uint32_t x = cnt;
#pragma unroll
    for (int q = 1; q < 32; q <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, q);
        if (lane >= q) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
    for (int w = 0; w < kDecThreads / 32; ++w) {
        if (w < warp) wbase += s_wsum[w];
        total += s_wsum[w];
    }
    // the block's count for its successors' look-back (its own prefix when first)
    if (tid == 0) st_volatile_u64(look + bid, (bid == 0 ? kFlagPre : kFlagAgg) | total);
    // the colour and covariance heads (BF16 form) while predecessors publish theirs
    if (p.bf16) {
        head(std::integral_constant<int, 1>{});
        head(std::integral_constant<int, 2>{});
    }
    // the (anchor, m) of each of the block's output slots, in (anchor, m) order
    {
        uint32_t at = wbase + (x - cnt);
        for (int m = 0; m < K; ++m)
            if (mask >> m & 1u) S.slot[at++] = (uint16_t)((tid << 4) | m);
    }
    __syncthreads();
    // every slot's head outputs turned into the Gaussian's values in place
    // (activations, normalised quaternion, mean), so that once the block's offset
    // is known the outputs are plain copies; then the decoupled look-back over
    // earlier blocks (one warp, 32 predecessors per step), which by now mostly
    // finds their counts published
    {
        for (uint32_t sl = tid; sl < total; sl += kDecThreads) {
            const uint32_t e = S.slot[sl];
            const int al = (int)(e >> 4), m = (int)(e & 15u);
            const int64_t aa = bid * kDecAnchors + al;
            float *orw = S.out + al * kOutStride;
            const float l0 = p.scaling[3 * aa], l1 = p.scaling[3 * aa + 1], l2 = p.scaling[3 * aa + 2];
            const float *O = p.offsets + (aa * K + m) * 3;
            float *mw = S.mean + al * 3 * kMaxK + 3 * m;
            mw[0] = fmaf(O[0], l0, p.anchors[3 * aa]);
            mw[1] = fmaf(O[1], l1, p.anchors[3 * aa + 1]);
            mw[2] = fmaf(O[2], l2, p.anchors[3 * aa + 2]);
            orw[kColOpa + m] = tanhf(orw[kColOpa + m]);
            float *cc = orw + kColCol + 3 * m;
            cc[0] = sigmoidf_(cc[0]);
            cc[1] = sigmoidf_(cc[1]);
            cc[2] = sigmoidf_(cc[2]);
            float *cv = orw + kColCov + 7 * m;
            cv[0] = sigmoidf_(cv[0]) * l0;
            cv[1] = sigmoidf_(cv[1]) * l1;
            cv[2] = sigmoidf_(cv[2]) * l2;
            const float inv = 1.0f / sqrtf(cv[3] * cv[3] + cv[4] * cv[4] + cv[5] * cv[5] + cv[6] * cv[6]);
            cv[3] *= inv;
            cv[4] *= inv;
            cv[5] *= inv;
            cv[6] *= inv;
        }
    }
    if (warp == 0) {
        unsigned long long excl = 0;
        if (bid != 0) {
            int64_t j0 = bid - 1;
            for (;;) {
                const int64_t j = j0 - lane;
                unsigned long long w = j >= 0 ? ld_volatile_u64(look + j) : kFlagPre;
                int spins = 0;
                bool timed_out = false;
                while (!__all_sync(0xffffffffu, (w >> 62) != 0)) {
                    if (++spins > kSpinLimit) {
                        timed_out = true;
                        break;
                    }
                    __nanosleep(64);
                    if ((w >> 62) == 0) w = ld_volatile_u64(look + j);
                }
                if (timed_out) {
                    if (lane == 0) set_status(status, VPGS_ERR_TIMEOUT);
                    break;
                }
                const uint32_t pre = __ballot_sync(0xffffffffu, (w >> 62) == 2);
                const int last = pre ? __ffs(pre) - 1 : 31;  // nearest inclusive prefix
                unsigned long long v = lane <= last ? (w & kValMask) : 0ull;
#pragma unroll
                for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
                excl += v;
                if (pre) break;
                j0 -= 32;
            }
            if (lane == 0) st_volatile_u64(look + bid, kFlagPre | (excl + total));
        }
        if (lane == 0) {
            s_base = (uint32_t)excl;
            s_total = total;
            if ((bid + 1) * kDecAnchors >= p.A) *o.n_out = (int32_t)(excl + total);
        }
    }
    __syncthreads();
    // one output Gaussian per thread, in output order
    const int64_t cap = p.A * K;
    const uint32_t tot = s_total;
    for (uint32_t sl = tid; sl < tot; sl += kDecThreads) {
        const int64_t pos = (int64_t)s_base + sl;
        if (pos >= cap) break;  // only after a timed-out look-back
        const uint32_t e = S.slot[sl];
        const int al = (int)(e >> 4), m = (int)(e & 15u);
        const int64_t aa = bid * kDecAnchors + al;
        const float *orw = S.out + al * kOutStride;
        const float *mw = S.mean + al * 3 * kMaxK + 3 * m;
        o.means[3 * pos] = mw[0];
        o.means[3 * pos + 1] = mw[1];
        o.means[3 * pos + 2] = mw[2];
        o.opac[pos] = orw[kColOpa + m];
        const float *cc = orw + kColCol + 3 * m;
        o.colors[3 * pos] = cc[0];
        o.colors[3 * pos + 1] = cc[1];
        o.colors[3 * pos + 2] = cc[2];
        const float *cv = orw + kColCov + 7 * m;
        o.scales[3 * pos] = cv[0];
        o.scales[3 * pos + 1] = cv[1];
        o.scales[3 * pos + 2] = cv[2];
        reinterpret_cast<float4 *>(o.quats)[pos] = make_float4(cv[3], cv[4], cv[5], cv[6]);
        o.src_index[pos] = (int32_t)(aa * K + m);
    }
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

__global__ void inverse_index_kernel(const int32_t *src_index, const int32_t *n_out, int64_t n_cap,
                                     int64_t inv_size, int32_t *inv) {
    grid_dep_enter();
    const int64_t n = min(n_cap, (int64_t)*n_out);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = src_index[i];
        if (s >= 0 && s < inv_size) inv[s] = (int32_t)i;
    }
}

struct DecGradIn {
    const float *means, *scales, *quats, *opac, *colors;
};

struct DecGradOut {
    float *features, *offsets, *scaling, *params;
};

constexpr int kBwdAnchors = 64;
constexpr int kRowIn = 37, kRowH = 33, kRowOut = 73;

struct DecBwdSmem {
    float w[8192];                                  // effective (FP32 or BF16-rounded) weights
    float in[kBwdAnchors * kRowIn];
    float h[kBwdAnchors * kRowH];
    float dpre[kBwdAnchors * kRowH];
    float dout[kBwdAnchors * kRowOut];
    float din[kBwdAnchors * kRowIn];
};

__global__ void __launch_bounds__(kBwdAnchors)
decode_bwd_kernel(DecParams p, const double *__restrict__ T, const int32_t *__restrict__ inv,
                  DecGradIn gin, DecGradOut gout) {
    grid_dep_enter();
    extern __shared__ __align__(16) unsigned char dsm[];
    DecBwdSmem &S = *reinterpret_cast<DecBwdSmem *>(dsm);
    __shared__ DecCam s_cam;
    const int tid = threadIdx.x;
    const int K = p.K;
    const int np = n_params(K);
    if (tid == 0) load_dec_cam(T, s_cam);
    for (int i = tid; i < np; i += kBwdAnchors) {
        // BF16 form: the weight matrices were rounded in the forward pass, biases were not
        float wv = p.params[i];
        if (p.bf16) {
            bool is_bias = false;
            for (int j = 0; j < 3; ++j) {
                const MlpOff m = mlp_off(K, j);
                if ((i >= m.b1 && i < m.b1 + kHid) || (i >= m.b2 && i < m.b2 + m.out)) is_bias = true;
            }
            if (!is_bias) wv = bf16r(wv);
        }
        S.w[i] = wv;
    }
    __syncthreads();
    const int64_t a = (int64_t)blockIdx.x * kBwdAnchors + tid;
    const bool live = a < p.A;
    float in[kIn];
    bool keep = false;
    if (live) keep = anchor_inputs(p, s_cam, a, in);
    float *sin_ = S.in + tid * kRowIn;
    float *sh = S.h + tid * kRowH;
    float *sdp = S.dpre + tid * kRowH;
    float *sdo = S.dout + tid * kRowOut;
    float *sdi = S.din + tid * kRowIn;
    for (int k = 0; k < kIn; ++k) {
        sin_[k] = keep ? in[k] : 0.f;
        sdi[k] = 0.f;
    }
    // which decoded Gaussians of this anchor survived, and where they are
    int idx[kMaxK];
    bool any = false;
    for (int m = 0; m < K; ++m) {
        idx[m] = keep ? inv[a * K + m] : -1;
        any |= idx[m] >= 0;
    }
    float l[3] = {0, 0, 0}, dl[3] = {0, 0, 0};
    if (live) {
        l[0] = p.scaling[3 * a]; l[1] = p.scaling[3 * a + 1]; l[2] = p.scaling[3 * a + 2];
    }
    for (int j = 0; j < 3; ++j) {
        const MlpOff m = mlp_off(K, j);
        // recompute hidden activations
        float h[kHid];
        for (int q = 0; q < kHid; ++q) {
            float acc = S.w[m.b1 + q];
            for (int k = 0; k < kIn; ++k) acc = fmaf(S.w[m.w1 + q * kIn + k], in[k], acc);
            const float hv = fmaxf(acc, 0.f);
            h[q] = p.bf16 ? bf16r(hv) : hv;
            sh[q] = any ? h[q] : 0.f;
            sdp[q] = acc > 0.f ? 1.f : 0.f;  // ReLU mask, turned into dpre below
        }
        float dh[kHid];
        for (int q = 0; q < kHid; ++q) dh[q] = 0.f;
        for (int n = 0; n < m.out; ++n) sdo[n] = 0.f;
        if (any) {
            for (int g = 0; g < K; ++g) {
                const int i = idx[g];
                if (i < 0) continue;
                // outputs of this Gaussian in MLP j
                const int w = j == 0 ? 1 : (j == 1 ? 3 : 7);
                float o[7];
                for (int r = 0; r < w; ++r) {
                    const int n = w * g + r;
                    float acc = S.w[m.b2 + n];
                    for (int k = 0; k < kHid; ++k) acc = fmaf(S.w[m.w2 + n * kHid + k], h[k], acc);
                    o[r] = acc;
                }
                float d[7];
                if (j == 0) {
                    const float al = tanhf(o[0]);
                    d[0] = gin.opac[i] * (1.f - al * al);
                } else if (j == 1) {
                    for (int r = 0; r < 3; ++r) {
                        const float c = sigmoidf_(o[r]);
                        d[r] = gin.colors[3 * i + r] * c * (1.f - c);
                    }
                } else {
                    for (int r = 0; r < 3; ++r) {
                        const float sg = sigmoidf_(o[r]);
                        const float gs = gin.scales[3 * i + r];
                        d[r] = gs * l[r] * sg * (1.f - sg);
                        dl[r] += gs * sg;
                    }
                    const float nrm = sqrtf(o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6]);
                    const float inn = 1.0f / nrm;
                    const float4 gq = reinterpret_cast<const float4 *>(gin.quats)[i];
                    const float qn[4] = {o[3] * inn, o[4] * inn, o[5] * inn, o[6] * inn};
                    const float gqv[4] = {gq.x, gq.y, gq.z, gq.w};
                    const float dot = qn[0] * gqv[0] + qn[1] * gqv[1] + qn[2] * gqv[2] + qn[3] * gqv[3];
                    for (int r = 0; r < 4; ++r) d[3 + r] = (gqv[r] - qn[r] * dot) * inn;
                }
                for (int r = 0; r < w; ++r) {
                    const int n = w * g + r;
                    sdo[n] = d[r];
                    for (int k = 0; k < kHid; ++k) dh[k] = fmaf(S.w[m.w2 + n * kHid + k], d[r], dh[k]);
                }
            }
        }
        float dpre[kHid];
        for (int q = 0; q < kHid; ++q) {
            dpre[q] = any ? dh[q] * sdp[q] : 0.f;
            sdp[q] = dpre[q];
        }
        for (int k = 0; k < kIn; ++k) {
            float acc = 0.f;
            for (int q = 0; q < kHid; ++q) acc = fmaf(S.w[m.w1 + q * kIn + k], dpre[q], acc);
            sdi[k] += acc;
        }
        __syncthreads();
        // block reduction of the weight gradients of MLP j
        if (gout.params) {
            for (int e = tid; e < kHid * kIn; e += kBwdAnchors) {  // dW1[q][k] = sum_a dpre[a][q] in[a][k]
                const int q = e / kIn, k = e % kIn;
                float acc = 0.f;
                for (int r = 0; r < kBwdAnchors; ++r) acc = fmaf(S.dpre[r * kRowH + q], S.in[r * kRowIn + k], acc);
                if (acc != 0.f) atomicAdd(gout.params + m.w1 + e, acc);
            }
            for (int q = tid; q < kHid; q += kBwdAnchors) {
                float acc = 0.f;
                for (int r = 0; r < kBwdAnchors; ++r) acc += S.dpre[r * kRowH + q];
                if (acc != 0.f) atomicAdd(gout.params + m.b1 + q, acc);
            }
            for (int e = tid; e < m.out * kHid; e += kBwdAnchors) {  // dW2[n][k] = sum_a dout[a][n] h[a][k]
                const int n = e / kHid, k = e % kHid;
                float acc = 0.f;
                for (int r = 0; r < kBwdAnchors; ++r) acc = fmaf(S.dout[r * kRowOut + n], S.h[r * kRowH + k], acc);
                if (acc != 0.f) atomicAdd(gout.params + m.w2 + e, acc);
            }
            for (int n = tid; n < m.out; n += kBwdAnchors) {
                float acc = 0.f;
                for (int r = 0; r < kBwdAnchors; ++r) acc += S.dout[r * kRowOut + n];
                if (acc != 0.f) atomicAdd(gout.params + m.b2 + n, acc);
            }
        }
        __syncthreads();
    }
    if (!live || !any) return;
    if (gout.features)
        for (int k = 0; k < kFeat; ++k) gout.features[kFeat * a + k] += sdi[k];
    for (int g = 0; g < K; ++g) {
        const int i = idx[g];
        if (i < 0) continue;
        const float *O = p.offsets + (a * K + g) * 3;
        const float gm[3] = {gin.means[3 * i], gin.means[3 * i + 1], gin.means[3 * i + 2]};
        for (int r = 0; r < 3; ++r) {
            if (gout.offsets) gout.offsets[(a * K + g) * 3 + r] += gm[r] * l[r];
            dl[r] += gm[r] * O[r];
        }
    }
    if (gout.scaling)
        for (int r = 0; r < 3; ++r) gout.scaling[3 * a + r] += dl[r];
}

// ---------------------------------------------------------------------------
// BF16 backward on tensor cores.  Persistent blocks of 256 threads walk chunks
// of 128 anchors; in the tensor-core phases each of the 8 warps owns one 16-row
// tile of anchors, in the per-anchor phases two threads serve each anchor
// (alternate Gaussians, halves of the features).  Per MLP:
//   P = In W1^T + b1 and O = H W2^T + b2 are recomputed with BF16 operands
//   (exact: inputs, weights and H are BF16 values), the head derivatives dO
//   are formed per anchor, then
//   dH = dO W2,  dPre = dH * [P > 0],  dIn += dPre W1,
//   dW1 += dPre^T [In | 1],  dW2 += dO^T [H | 1]   (the ones give db1, db2).
// dO and dPre are FP32; they enter the MMAs as hi + lo BF16 pairs (relative
// error 2^-16 per term) with FP32 accumulation.  Weight gradients accumulate in
// shared memory over the block's chunks and reach global memory once per block.
// ---------------------------------------------------------------------------
constexpr int kMA = 128;                 // anchors per chunk
constexpr int kMT = 2 * kMA;             // threads: two per anchor, 16 chunk rows per warp
constexpr int kAS = kMA + 8;             // row stride (bf16) of anchor-major staging
constexpr int kOS = 81;                  // row stride (float) of per-anchor output rows
constexpr int kW2T = 88;                 // row stride (bf16) of W2^T rows (outputs padded to 80)
constexpr int kW1T = 40;                 // row stride (bf16) of W1^T rows (hidden 32 + pad)
constexpr int kGW = 40;                  // columns of the weight-gradient accumulators
VPGS_HD int out_pad16(int j) { return j == 0 ? 16 : (j == 1 ? 32 : 80); }  // per-MLP outputs padded to 16
VPGS_HD int out_base(int j) { return j == 0 ? 0 : (j == 1 ? 16 : 48); }    // rows of MLP j in W2 / dW2 (K <= 10)

// The backward's effective weights (BF16-rounded matrices, FP32 biases) in
// the four layouts its MMAs read; prepared once per call by
// decode_bwd_weights_kernel and copied into each block's shared memory as
// 16-byte words.
struct DecBwdWts {
    __nv_bfloat16 w1[96 * kInPad];       // [hid][in]  (forward layout)
    __nv_bfloat16 w2[120 * kW2Pad];      // [out][hid] (forward layout)
    __nv_bfloat16 w2t[96 * kW2T];        // [MLP*32 + hid][out]
    __nv_bfloat16 w1t[3 * 40 * kW1T];    // [MLP][in][hid]
    float b1[96], b2[120];
};
static_assert(sizeof(DecBwdWts) % 16 == 0 && sizeof(DecBwdWts) <= kDecWtsBytes, "prepared weights: 16-byte words");

struct DecBwdMmaSmem {
    DecBwdWts wt;
    __nv_bfloat16 inrow[kMA * kInPad];   // [anchor][in]
    __nv_bfloat16 inT[40 * kAS];         // [in | 1 | 0][anchor]
    __nv_bfloat16 hT[40 * kAS];          // [hid | 1 | 0][anchor]
    __nv_bfloat16 dpT[2][32 * kAS];      // dPre^T hi / lo: [hid][anchor]
    __nv_bfloat16 doT[2][80 * kAS];      // dO^T hi / lo: [out][anchor]
    float orow[kMA * kOS];               // per anchor: O, then dO, finally dIn
    float gw1[3 * 32 * kGW];             // dW1 | db1 per MLP
    float gw2[128 * kGW];                // dW2 | db2, rows out_base(j) + out
};

VPGS_D void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// A fragment pair (hi, lo) of two FP32 values
VPGS_D void pack_split(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(x0, h0, l0);
    split_bf16(x1, h1, l1);
    __nv_bfloat162 H = __halves2bfloat162(h0, h1), L = __halves2bfloat162(l0, l1);
    hi = *reinterpret_cast<uint32_t *>(&H);
    lo = *reinterpret_cast<uint32_t *>(&L);
}

VPGS_D uint32_t ld_u32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__global__ void __launch_bounds__(256) decode_bwd_weights_kernel(DecParams p, DecBwdWts *wts) {
    grid_dep_enter();
    const int K = p.K, tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int i = tid; i < 96 * kInPad; i += stride) {
        const int r = i / kInPad, c = i % kInPad;
        wts->w1[i] = __float2bfloat16_rn(c < kIn ? p.params[mlp_off(K, r / 32).w1 + (r % 32) * kIn + c] : 0.f);
    }
    for (int i = tid; i < 120 * kW2Pad; i += stride) {
        const int r = i / kW2Pad, c = i % kW2Pad;
        const int j = r < kColCol ? 0 : (r < kColCov ? 1 : 2);
        const MlpOff m = mlp_off(K, j);
        const int n = r - out_base(j);
        wts->w2[i] = __float2bfloat16_rn((c < kHid && n < m.out) ? p.params[m.w2 + n * kHid + c] : 0.f);
    }
    for (int i = tid; i < 96 * kW2T; i += stride) {
        const int r = i / kW2T, n = i % kW2T, j = r / 32, q = r % 32;
        const MlpOff m = mlp_off(K, j);
        wts->w2t[i] = __float2bfloat16_rn(n < m.out ? p.params[m.w2 + n * kHid + q] : 0.f);
    }
    for (int i = tid; i < 3 * 40 * kW1T; i += stride) {
        const int j = i / (40 * kW1T), rem = i % (40 * kW1T), k = rem / kW1T, q = rem % kW1T;
        wts->w1t[i] = __float2bfloat16_rn((k < kIn && q < kHid) ? p.params[mlp_off(K, j).w1 + q * kIn + k] : 0.f);
    }
    for (int i = tid; i < 96; i += stride) wts->b1[i] = p.params[mlp_off(K, i / 32).b1 + i % 32];
    for (int i = tid; i < 120; i += stride) {
        const int j = i < kColCol ? 0 : (i < kColCov ? 1 : 2);
        const MlpOff m = mlp_off(K, j);
        wts->b2[i] = (i - out_base(j) < m.out) ? p.params[m.b2 + i - out_base(j)] : 0.f;
    }
}

__global__ void __launch_bounds__(kMT, 1)
decode_bwd_mma_kernel(DecParams p, const double *__restrict__ T, const int32_t *__restrict__ inv,
                      const DecBwdWts *__restrict__ wts, DecGradIn gin, DecGradOut gout) {
    grid_dep_enter();
    extern __shared__ __align__(16) unsigned char dsm[];
    DecBwdMmaSmem &S = *reinterpret_cast<DecBwdMmaSmem *>(dsm);
    __shared__ DecCam s_cam;
    __shared__ float s_dl[kMA][3];
    __shared__ uint8_t s_keep[kMA];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int K = p.K;
    if (tid == 0) load_dec_cam(T, s_cam);
    {
        // the prepared weights into shared memory, 16-byte words
        const uint4 *src = reinterpret_cast<const uint4 *>(wts);
        uint4 *dst = reinterpret_cast<uint4 *>(&S.wt);
        for (int i = tid; i < (int)(sizeof(DecBwdWts) / 16); i += kMT) dst[i] = src[i];
    }
    // constant rows: the ones that turn the weight-gradient products into bias gradients
    for (int i = tid; i < 4 * kAS; i += kMT) {
        const __nv_bfloat16 v = __float2bfloat16_rn(i < kAS ? 1.f : 0.f);
        S.inT[36 * kAS + i] = v;
        S.hT[32 * kAS + i] = v;
        S.hT[36 * kAS + i] = __float2bfloat16_rn(0.f);
    }
    for (int i = tid; i < 3 * 32 * kGW; i += kMT) S.gw1[i] = 0.f;
    for (int i = tid; i < 128 * kGW; i += kMT) S.gw2[i] = 0.f;
    __syncthreads();

    // work: full chunks of kMA anchors in whole rounds over the grid, then the
    // anchors left over split evenly into one short chunk per block (rows past
    // its length are masked), so that the last round leaves no block idle
    const int64_t full = (p.A / kMA) / gridDim.x * gridDim.x;
    const int64_t rest = p.A - full * kMA;
    const int64_t unit = rest > 0 ? min((int64_t)kMA, (rest + gridDim.x - 1) / gridDim.x) : 1;
    const int64_t n_work = full + (rest + unit - 1) / unit;
    // the anchor row this thread serves in the per-anchor phases (two threads per
    // anchor), and the warp's 16 chunk rows in the tensor-core phases
    const int ta = tid & (kMA - 1), half = tid / kMA;
    const int r0 = warp * 16;
    for (int64_t wk = blockIdx.x; wk < n_work; wk += gridDim.x) {
        const int64_t base = wk < full ? wk * kMA : full * kMA + (wk - full) * unit;
        const int64_t rows = wk < full ? (int64_t)kMA : min(unit, p.A - base);
        // ---- per anchor: inputs (first thread of the pair), surviving Gaussians
        const int64_t a = base + ta;
        const bool live = ta < rows && a < p.A;
        if (half == 0) {
            float in[kIn];
            bool kp = false;
            if (live) kp = anchor_inputs(p, s_cam, a, in);
            for (int k = 0; k < kInPad; ++k) {
                const __nv_bfloat16 v = __float2bfloat16_rn(kp && k < kIn ? in[k] : 0.f);
                S.inrow[ta * kInPad + k] = v;
                if (k < kIn) S.inT[k * kAS + ta] = v;
            }
            s_keep[ta] = kp ? 1 : 0;
        }
        float l[3] = {0, 0, 0}, dl[3] = {0, 0, 0};
        if (live) {
            l[0] = p.scaling[3 * a]; l[1] = p.scaling[3 * a + 1]; l[2] = p.scaling[3 * a + 2];
        }
        float dIn[5][4];
#pragma unroll
        for (int nt = 0; nt < 5; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) dIn[nt][e] = 0.f;
        __syncthreads();
        const bool keep = s_keep[ta] != 0;
        int idx[kMaxK];
        bool any = false;
        for (int m = 0; m < K; ++m) {
            idx[m] = keep ? inv[a * K + m] : -1;
            any |= idx[m] >= 0;
        }
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            const int ntl2 = j == 0 ? 2 : (j == 1 ? 4 : 9);
            const int kd_steps = out_pad16(j) / 16;
            uint32_t mask = 0u;
            // ---- layer 1 and 2 on tensor cores (rows r0 .. r0 + 15 of the chunk)
            {
                float acc[4][4];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const float b0 = S.wt.b1[32 * j + 8 * nt + 2 * t4], b1v = S.wt.b1[32 * j + 8 * nt + 2 * t4 + 1];
                    acc[nt][0] = b0; acc[nt][1] = b1v; acc[nt][2] = b0; acc[nt][3] = b1v;
                }
                const __nv_bfloat16 *A0 = S.inrow + (r0 + g) * kInPad, *A1 = S.inrow + (r0 + g + 8) * kInPad;
#pragma unroll
                for (int ks = 0; ks < 3; ++ks) {
                    const int c0 = 16 * ks + 2 * t4;
                    const uint32_t a0 = ld_u32(A0 + c0), a1 = ld_u32(A1 + c0), a2 = ld_u32(A0 + c0 + 8),
                                   a3 = ld_u32(A1 + c0 + 8);
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) {
                        const __nv_bfloat16 *B = S.wt.w1 + (32 * j + 8 * nt + g) * kInPad;
                        mma_bf16_16816(acc[nt], a0, a1, a2, a3, ld_u32(B + c0), ld_u32(B + c0 + 8));
                    }
                }
                // ReLU mask, H (BF16) into hT and as layer-2 A fragments
                uint32_t ha[2][4];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (acc[nt][e] > 0.f) mask |= 1u << (4 * nt + e);
                        const int q = 8 * nt + 2 * t4 + (e & 1), row = r0 + g + 8 * (e >> 1);
                        S.hT[q * kAS + row] = __float2bfloat16_rn(fmaxf(acc[nt][e], 0.f));
                    }
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const float *x0 = acc[2 * kk], *x1 = acc[2 * kk + 1];
                    ha[kk][0] = pack_bf16(fmaxf(x0[0], 0.f), fmaxf(x0[1], 0.f));
                    ha[kk][1] = pack_bf16(fmaxf(x0[2], 0.f), fmaxf(x0[3], 0.f));
                    ha[kk][2] = pack_bf16(fmaxf(x1[0], 0.f), fmaxf(x1[1], 0.f));
                    ha[kk][3] = pack_bf16(fmaxf(x1[2], 0.f), fmaxf(x1[3], 0.f));
                }
                for (int nt = 0; nt < ntl2; ++nt) {
                    const int col = out_base(j) + 8 * nt + 2 * t4;
                    float d[4] = {S.wt.b2[col], S.wt.b2[col + 1], S.wt.b2[col], S.wt.b2[col + 1]};
                    const __nv_bfloat16 *B = S.wt.w2 + (out_base(j) + 8 * nt + g) * kW2Pad;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const int c0 = 16 * kk + 2 * t4;
                        mma_bf16_16816(d, ha[kk][0], ha[kk][1], ha[kk][2], ha[kk][3], ld_u32(B + c0),
                                       ld_u32(B + c0 + 8));
                    }
                    const int lc = 8 * nt + 2 * t4;
                    S.orow[(r0 + g) * kOS + lc] = d[0];
                    S.orow[(r0 + g) * kOS + lc + 1] = d[1];
                    S.orow[(r0 + g + 8) * kOS + lc] = d[2];
                    S.orow[(r0 + g + 8) * kOS + lc + 1] = d[3];
                }
            }
            __syncthreads();
            // ---- per anchor: head derivatives dO (0 where no Gaussian survived); the
            // pair's two threads take alternate Gaussians, each reading its outputs
            // before overwriting them with their derivatives
            {
                float *orw = S.orow + ta * kOS;
                auto put = [&](int n, float v) {
                    orw[n] = v;
                    split_bf16(v, S.doT[0][n * kAS + ta], S.doT[1][n * kAS + ta]);
                };
                for (int gm = half; gm < K; gm += 2) {
                    const int i = idx[gm];
                    if (j == 0) {
                        float v = 0.f;
                        if (i >= 0) {
                            const float al = tanhf(orw[gm]);
                            v = gin.opac[i] * (1.f - al * al);
                        }
                        put(gm, v);
                    } else if (j == 1) {
                        float o[3];
#pragma unroll
                        for (int r = 0; r < 3; ++r) o[r] = orw[3 * gm + r];
#pragma unroll
                        for (int r = 0; r < 3; ++r) {
                            float v = 0.f;
                            if (i >= 0) {
                                const float c = sigmoidf_(o[r]);
                                v = gin.colors[3 * i + r] * c * (1.f - c);
                            }
                            put(3 * gm + r, v);
                        }
                    } else {
                        float o[7];
#pragma unroll
                        for (int r = 0; r < 7; ++r) o[r] = orw[7 * gm + r];
                        float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        if (i >= 0) {
#pragma unroll
                            for (int r = 0; r < 3; ++r) {
                                const float sg = sigmoidf_(o[r]);
                                const float gs = gin.scales[3 * i + r];
                                v[r] = gs * l[r] * sg * (1.f - sg);
                                dl[r] += gs * sg;
                            }
                            const float nrm = sqrtf(o[3] * o[3] + o[4] * o[4] + o[5] * o[5] + o[6] * o[6]);
                            const float inn = 1.0f / nrm;
                            const float4 gq = reinterpret_cast<const float4 *>(gin.quats)[i];
                            const float qn[4] = {o[3] * inn, o[4] * inn, o[5] * inn, o[6] * inn};
                            const float gqv[4] = {gq.x, gq.y, gq.z, gq.w};
                            const float dot = qn[0] * gqv[0] + qn[1] * gqv[1] + qn[2] * gqv[2] + qn[3] * gqv[3];
#pragma unroll
                            for (int r = 0; r < 4; ++r) v[3 + r] = (gqv[r] - qn[r] * dot) * inn;
                        }
#pragma unroll
                        for (int r = 0; r < 7; ++r) put(7 * gm + r, v[r]);
                    }
                }
                if (half == 0) {  // the padding columns of the 16-wide output tiles
                    const int w = j == 0 ? 1 : (j == 1 ? 3 : 7);
                    for (int n = w * K; n < out_pad16(j); ++n) put(n, 0.f);
                }
            }
            __syncthreads();
            // ---- dH = dO W2, dPre = dH [P > 0], dIn += dPre W1, dPre^T staged
            {
                float dh[4][4];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) dh[nt][e] = 0.f;
                const float *O0 = S.orow + (r0 + g) * kOS, *O1 = S.orow + (r0 + g + 8) * kOS;
                for (int kd = 0; kd < kd_steps; ++kd) {
                    const int c0 = 16 * kd + 2 * t4;
                    uint32_t ah[4], alo[4];
                    pack_split(O0[c0], O0[c0 + 1], ah[0], alo[0]);
                    pack_split(O1[c0], O1[c0 + 1], ah[1], alo[1]);
                    pack_split(O0[c0 + 8], O0[c0 + 9], ah[2], alo[2]);
                    pack_split(O1[c0 + 8], O1[c0 + 9], ah[3], alo[3]);
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) {
                        const __nv_bfloat16 *B = S.wt.w2t + (32 * j + 8 * nt + g) * kW2T;
                        const uint32_t b0 = ld_u32(B + c0), b1 = ld_u32(B + c0 + 8);
                        mma_bf16_16816(dh[nt], ah[0], ah[1], ah[2], ah[3], b0, b1);
                        mma_bf16_16816(dh[nt], alo[0], alo[1], alo[2], alo[3], b0, b1);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (!(mask >> (4 * nt + e) & 1u)) dh[nt][e] = 0.f;
                        const int q = 8 * nt + 2 * t4 + (e & 1), row = r0 + g + 8 * (e >> 1);
                        split_bf16(dh[nt][e], S.dpT[0][q * kAS + row], S.dpT[1][q * kAS + row]);
                    }
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    uint32_t ah[4], alo[4];
                    const float *x0 = dh[2 * kk], *x1 = dh[2 * kk + 1];
                    pack_split(x0[0], x0[1], ah[0], alo[0]);
                    pack_split(x0[2], x0[3], ah[1], alo[1]);
                    pack_split(x1[0], x1[1], ah[2], alo[2]);
                    pack_split(x1[2], x1[3], ah[3], alo[3]);
                    const int c0 = 16 * kk + 2 * t4;
#pragma unroll
                    for (int nt = 0; nt < 5; ++nt) {
                        const __nv_bfloat16 *B = S.wt.w1t + (j * 40 + 8 * nt + g) * kW1T;
                        const uint32_t b0 = ld_u32(B + c0), b1 = ld_u32(B + c0 + 8);
                        mma_bf16_16816(dIn[nt], ah[0], ah[1], ah[2], ah[3], b0, b1);
                        mma_bf16_16816(dIn[nt], alo[0], alo[1], alo[2], alo[3], b0, b1);
                    }
                }
            }
            __syncthreads();
            // ---- weight gradients of MLP j over the chunk's anchors
            if (gout.params) {
                const int mt2 = out_pad16(j) / 16;
                const int n1 = 2 * 5, n2 = mt2 * 5;
                for (int t = warp; t < n1 + n2; t += kMT / 32) {
                    const bool first = t < n1;
                    const int tt = first ? t : t - n1;
                    const int mt = tt / 5, nt = tt % 5;
                    const __nv_bfloat16 *Ah = first ? S.dpT[0] : S.doT[0];
                    const __nv_bfloat16 *Al = first ? S.dpT[1] : S.doT[1];
                    const __nv_bfloat16 *Bm = first ? S.inT : S.hT;
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    const int ra = (16 * mt + g) * kAS, rb = (16 * mt + g + 8) * kAS, rB = (8 * nt + g) * kAS;
#pragma unroll 4
                    for (int ks = 0; ks < kMA / 16; ++ks) {
                        const int c0 = 16 * ks + 2 * t4;
                        const uint32_t b0 = ld_u32(Bm + rB + c0), b1 = ld_u32(Bm + rB + c0 + 8);
                        mma_bf16_16816(acc, ld_u32(Ah + ra + c0), ld_u32(Ah + rb + c0), ld_u32(Ah + ra + c0 + 8),
                                       ld_u32(Ah + rb + c0 + 8), b0, b1);
                        mma_bf16_16816(acc, ld_u32(Al + ra + c0), ld_u32(Al + rb + c0), ld_u32(Al + ra + c0 + 8),
                                       ld_u32(Al + rb + c0 + 8), b0, b1);
                    }
                    float *G = first ? S.gw1 + j * 32 * kGW : S.gw2 + out_base(j) * kGW;
                    const int c = 8 * nt + 2 * t4;
                    G[(16 * mt + g) * kGW + c] += acc[0];
                    G[(16 * mt + g) * kGW + c + 1] += acc[1];
                    G[(16 * mt + g + 8) * kGW + c] += acc[2];
                    G[(16 * mt + g + 8) * kGW + c + 1] += acc[3];
                }
            }
            __syncthreads();
        }
        // ---- dIn rows, then per anchor: feature, offset and scaling gradients
#pragma unroll
        for (int nt = 0; nt < 5; ++nt) {
            const int c = 8 * nt + 2 * t4;
            S.orow[(r0 + g) * kOS + c] = dIn[nt][0];
            S.orow[(r0 + g) * kOS + c + 1] = dIn[nt][1];
            S.orow[(r0 + g + 8) * kOS + c] = dIn[nt][2];
            S.orow[(r0 + g + 8) * kOS + c + 1] = dIn[nt][3];
        }
        __syncthreads();
        if (live && any) {
            // the pair splits the features in halves and the Gaussians by parity
            if (gout.features)
                for (int k = half * (kFeat / 2); k < (half + 1) * (kFeat / 2); ++k)
                    gout.features[kFeat * a + k] += S.orow[ta * kOS + k];
            for (int gm = half; gm < K; gm += 2) {
                const int i = idx[gm];
                if (i < 0) continue;
                const float *O = p.offsets + (a * K + gm) * 3;
                const float gmn[3] = {gin.means[3 * i], gin.means[3 * i + 1], gin.means[3 * i + 2]};
                for (int r = 0; r < 3; ++r) {
                    if (gout.offsets) gout.offsets[(a * K + gm) * 3 + r] += gmn[r] * l[r];
                    dl[r] += gmn[r] * O[r];
                }
            }
        }
        if (half == 1) {
            s_dl[ta][0] = dl[0];
            s_dl[ta][1] = dl[1];
            s_dl[ta][2] = dl[2];
        }
        __syncthreads();
        if (half == 0 && live && any && gout.scaling)
            for (int r = 0; r < 3; ++r) gout.scaling[3 * a + r] += dl[r] + s_dl[ta][r];
        __syncthreads();  // orow, the staging rows and s_dl are rewritten by the next chunk
    }
    // ---- the block's weight gradients, once
    if (gout.params) {
        for (int i = tid; i < 3 * 32 * kGW; i += kMT) {
            const int j = i / (32 * kGW), q = (i / kGW) % 32, c = i % kGW;
            const MlpOff m = mlp_off(K, j);
            const float v = S.gw1[i];
            if (v == 0.f) continue;
            if (c < kIn) atomicAdd(gout.params + m.w1 + q * kIn + c, v);
            else if (c == kIn) atomicAdd(gout.params + m.b1 + q, v);
        }
        for (int i = tid; i < 128 * kGW; i += kMT) {
            const int r = i / kGW, c = i % kGW;
            const int j = r < kColCol ? 0 : (r < kColCov ? 1 : 2);
            const MlpOff m = mlp_off(K, j);
            const int n = r - out_base(j);
            const float v = S.gw2[i];
            if (v == 0.f || n >= m.out) continue;
            if (c < kHid) atomicAdd(gout.params + m.w2 + n * kHid + c, v);
            else if (c == kHid) atomicAdd(gout.params + m.b2 + n, v);
        }
    }
}

// ---------------------------------------------------------------------------
// workspace: [0] status, [256] counters (ticket), [512] look-back words, inverse map
// ---------------------------------------------------------------------------
struct DecLayout {
    size_t off_status, off_counters, off_look, off_inv, off_wts, total;
    int64_t nblocks;
};

static DecLayout dec_layout(int64_t A, int K) {
    DecLayout L;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    L.nblocks = (A + kDecAnchors - 1) / kDecAnchors;
    L.off_status = 0;
    L.off_counters = 256;
    L.off_look = 512;
    L.off_inv = up(L.off_look + 8 * (size_t)std::max<int64_t>(L.nblocks, 1));
    L.off_wts = up(L.off_inv + 4 * (size_t)std::max<int64_t>(A * K, 1));
    L.total = up(L.off_wts + kDecWtsBytes);
    return L;
}

static bool fill_params(const vpgs_anchors *a, const vpgs_mlp *mlp, const vpgs_camera *cam,
                        const vpgs_decode_opts *opts, DecParams &p) {
    if (!a || !mlp || !cam || !opts || !mlp->params || a->n < 0 || a->k < 1 || a->k > kMaxK) return false;
    if (a->n > 0 && (!a->anchors || !a->scaling || !a->offsets || !a->features)) return false;
    if (a->n * a->k >= (int64_t(1) << 31)) return false;
    if (cam->width <= 0 || cam->height <= 0) return false;
    if (!a->features_bf16 && (reinterpret_cast<uintptr_t>(a->features) & 15u)) return false;
    p.anchors = a->anchors; p.scaling = a->scaling; p.offsets = a->offsets; p.features = a->features;
    p.A = a->n; p.K = a->k; p.feat_bf16 = a->features_bf16 != 0;
    p.params = mlp->params; p.bf16 = mlp->bf16 != 0;
    p.fx = cam->fx; p.fy = cam->fy; p.cx = cam->cx; p.cy = cam->cy; p.W = cam->width; p.H = cam->height;
    p.near_z = opts->near_z; p.guard = opts->guard;
    return true;
}

}  // namespace vpgs

using namespace vpgs;

extern "C" {

size_t vpgs_decode_workspace_bytes(int64_t n_anchors, int32_t k) {
    if (n_anchors < 0 || k < 1 || k > kMaxK) return 0;
    return dec_layout(n_anchors, k).total;
}

vpgs_status vpgs_decode_anchors(void *ws, size_t ws_bytes, const vpgs_anchors *a, const vpgs_mlp *mlp,
                                const vpgs_camera *cam, const double *T_cw, const vpgs_decode_opts *opts,
                                const vpgs_gaussian_buffers *out, int32_t *n_out, int32_t *src_index,
                                vpgs_stream stream) {
    DecParams p;
    if (!ws || !T_cw || !out || !n_out || !src_index || !fill_params(a, mlp, cam, opts, p))
        return VPGS_ERR_INVALID_ARG;
    if (!out->means || !out->scales || !out->quats || !out->opacities || !out->colors)
        return VPGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(out->quats) & 15u) return VPGS_ERR_INVALID_ARG;
    const DecLayout L = dec_layout(p.A, p.K);
    if (ws_bytes < L.total) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *b = static_cast<char *>(ws);
    cudaError_t e = cudaMemsetAsync(b, 0, L.off_look + 8 * (size_t)std::max<int64_t>(L.nblocks, 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_out, 0, sizeof(int32_t), s);
    if (e != cudaSuccess || p.A == 0) return e == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
    // the shared-memory opt-in is a per-device attribute: set on every call, on the current device
    const size_t smem = sizeof(DecFwdSmem);
    cudaFuncSetAttribute((const void *)decode_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    DecOut o{out->means, out->scales, out->quats, out->opacities, out->colors, n_out, src_index};
    uint32_t *status = reinterpret_cast<uint32_t *>(b + L.off_status);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(b + L.off_counters + 4 * CNT_TICKET_A);
    unsigned long long *look = reinterpret_cast<unsigned long long *>(b + L.off_look);
    DecWts *wts = reinterpret_cast<DecWts *>(b + L.off_wts);
    VPGS_LAUNCH("decode_weights", s, launch_k(decode_weights_kernel, 8, 256, 0, s, p, wts));
    // resident blocks only: each takes chunks from the ticket until none is left
    static std::atomic<int> fwd_cache[kDeviceCache];
    const int resident = per_device(fwd_cache, [smem] {
        return resident_grid((const void *)decode_fwd_kernel, kDecThreads, smem, int64_t(1) << 30);
    });
    const unsigned grid = (unsigned)std::min<int64_t>(L.nblocks, resident);
    VPGS_LAUNCH("decode_fwd", s,
                launch_k(decode_fwd_kernel, grid, kDecThreads, smem, s, p, T_cw, o,
                         (const DecWts *)wts, ticket, look, status));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

vpgs_status vpgs_decode_anchors_bwd(void *ws, size_t ws_bytes, const vpgs_anchors *a, const vpgs_mlp *mlp,
                                    const vpgs_camera *cam, const double *T_cw,
                                    const vpgs_decode_opts *opts, const vpgs_gaussians *dL,
                                    const int32_t *src_index, float *dL_dfeatures, float *dL_doffsets,
                                    float *dL_dscaling, float *dL_dparams, vpgs_stream stream) {
    DecParams p;
    if (!ws || !T_cw || !dL || !src_index || !dL->n_dev || !fill_params(a, mlp, cam, opts, p))
        return VPGS_ERR_INVALID_ARG;
    if (!dL->means || !dL->scales || !dL->quats || !dL->opacities || !dL->colors)
        return VPGS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(dL->quats) & 15u) return VPGS_ERR_INVALID_ARG;
    const DecLayout L = dec_layout(p.A, p.K);
    if (ws_bytes < L.total) return VPGS_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p.A == 0) return VPGS_OK;
    char *b = static_cast<char *>(ws);
    int32_t *inv = reinterpret_cast<int32_t *>(b + L.off_inv);
    const int64_t cap = p.A * p.K;
    cudaError_t e = cudaMemsetAsync(inv, 0xff, 4 * (size_t)cap, s);
    if (e != cudaSuccess) return VPGS_ERR_CUDA;
    const int sms = device_sm_count();
    const int ib = (int)std::min<int64_t>((cap + 255) / 256, (int64_t)sms * 8);
    VPGS_LAUNCH("decode_inverse_index", s,
                launch_k(inverse_index_kernel, ib, 256, 0, s, src_index, dL->n_dev, dL->n, cap, inv));
    // the shared-memory opt-in is a per-device attribute: set on every call, on the current device
    const size_t smem = sizeof(DecBwdSmem);
    cudaFuncSetAttribute((const void *)decode_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    DecGradIn gin{dL->means, dL->scales, dL->quats, dL->opacities, dL->colors};
    DecGradOut gout{dL_dfeatures, dL_doffsets, dL_dscaling, dL_dparams};
    if (p.bf16 && VPGS_DECODE_BWD_MMA) {
        const size_t msm = sizeof(DecBwdMmaSmem);
        cudaFuncSetAttribute((const void *)decode_bwd_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)msm);
        const int64_t nch = (p.A + kMA - 1) / kMA;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nch, sms));
        DecBwdWts *wts = reinterpret_cast<DecBwdWts *>(b + L.off_wts);
        VPGS_LAUNCH("decode_bwd_weights", s, launch_k(decode_bwd_weights_kernel, 8, 256, 0, s, p, wts));
        VPGS_LAUNCH("decode_bwd", s, launch_k(decode_bwd_mma_kernel, grid, kMT, msm, s, p, T_cw, inv,
                                              (const DecBwdWts *)wts, gin, gout));
        return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
    }
    const unsigned nb = (unsigned)((p.A + kBwdAnchors - 1) / kBwdAnchors);
    VPGS_LAUNCH("decode_bwd", s, launch_k(decode_bwd_kernel, nb, kBwdAnchors, smem, s, p, T_cw, inv, gin, gout));
    return cudaGetLastError() == cudaSuccess ? VPGS_OK : VPGS_ERR_CUDA;
}

}  // extern "C"
