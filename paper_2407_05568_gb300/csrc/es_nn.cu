// es_nn.cu -- kernels of the learned mesh warm start: 3x3 convolution layers with
// BF16 weights and FP32 activations/accumulation, their backward passes, the MSE
// loss and the Adam update.  The network maps the filtered monitor, the
// fundamental derivative and the current mesh (Sec. 4) to the displacement that
// starts the Jacobi iteration; the plain iteration always finishes the solve.
//
// Layout: activations [B][C][H][W] float; weights [Cout][Cin][3][3] (bf16 in the
// C ABI, float inside the context); cross-correlation with zero padding:
//   out[co](y, x) = bias[co] + sum_{ci, dy, dx} w[co][ci][dy+1][dx+1] in[ci](y+dy, x+dx).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "es_internal.h"
#include "es_vdw.h"

namespace es {
namespace {

constexpr int TS = 16;            // output tile edge (pixels)
constexpr int HALO = TS + 2;
constexpr int MAXC = 32;          // channel limit
constexpr int WG_THREADS = 288;   // weight-gradient block: 9 * 32 (ci, tap) pairs

// One thread per output pixel with all COUT channels in registers.  The input tile
// with its halo and the weights (transposed to [ci][tap][co], so one thread reads
// COUT consecutive floats) sit in shared memory.
template <int COUT>
__global__ void __launch_bounds__(TS * TS) k_conv_fwd(const float* __restrict__ in, const float* __restrict__ wf,
                                                     const float* __restrict__ bias, float* __restrict__ out,
                                                     int Cin, int H, int W, int act) {
    extern __shared__ float4 sm4[];
    float* sm = reinterpret_cast<float*>(sm4);
    float* ws = sm;                                   // Cin * 9 * COUT
    float* xs = sm + COUT * Cin * 9;                  // Cin * HALO * HALO
    const int tx = threadIdx.x % TS, ty = threadIdx.x / TS;
    const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS, b = blockIdx.z;
    const size_t HW = size_t(H) * W;
    for (int k = threadIdx.x; k < COUT * Cin * 9; k += TS * TS) {
        const int co = k / (Cin * 9), r = k % (Cin * 9);
        ws[r * COUT + co] = wf[k];
    }
    const float* inb = in + size_t(b) * Cin * HW;
    for (int k = threadIdx.x; k < Cin * HALO * HALO; k += TS * TS) {
        const int ci = k / (HALO * HALO), r = k % (HALO * HALO);
        const int yy = y0 - 1 + r / HALO, xx = x0 - 1 + r % HALO;
        xs[k] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? inb[ci * HW + size_t(yy) * W + xx] : 0.0f;
    }
    __syncthreads();
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.0f;
    for (int ci = 0; ci < Cin; ++ci) {
        const float* xc = xs + ci * HALO * HALO + ty * HALO + tx;
        const float* wc = ws + ci * 9 * COUT;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = xc[(k / 3) * HALO + k % 3];
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[co] = fmaf(wc[k * COUT + co], v, acc[co]);
        }
    }
    const int x = x0 + tx, y = y0 + ty;
    if (x < W && y < H) {
        float* ob = out + size_t(b) * COUT * HW + size_t(y) * W + x;
#pragma unroll
        for (int co = 0; co < COUT; ++co) ob[co * HW] = act ? tanhf(acc[co]) : acc[co];
    }
}

// Weight and bias gradients of one strip of tiles (a 16-pixel column, `rows` tiles
// high, one image): thread (group gi, pair q = (ci, tap)) sums g[co](p) in[ci](p + tap)
// over its share of the strip's pixels for all COUT channels; the groups are summed in
// shared memory and the strip's partial sums written to partial[strip][...] (reduced
// over strips, in a fixed order, by k_reduce_partials).
template <int COUT>
__global__ void __launch_bounds__(WG_THREADS) k_conv_wgrad(const float* __restrict__ in,
                                                          const float* __restrict__ g, float* __restrict__ partial,
                                                          int Cin, int H, int W, int rows) {
    extern __shared__ float4 sm4[];
    float* sm = reinterpret_cast<float*>(sm4);
    float* gs = sm;                                   // TS*TS * COUT, [p][co]
    float* xs = sm + TS * TS * COUT;                  // Cin * HALO * HALO
    const int npairs = Cin * 9;
    const int G = WG_THREADS / npairs;                // pixel groups (Cin divides 32)
    const int q = threadIdx.x % npairs, gi = threadIdx.x / npairs;
    const int ci = q / 9, tap = q % 9;
    const int x0 = blockIdx.x * TS, b = blockIdx.z;
    const size_t HW = size_t(H) * W;
    const float* inb = in + size_t(b) * Cin * HW;
    const float* gb = g + size_t(b) * COUT * HW;
    float acc[COUT];
    float accb = 0.0f;                                // bias: threads 0..COUT-1
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.0f;
    for (int r = 0; r < rows; ++r) {
        const int y0 = (blockIdx.y * rows + r) * TS;
        if (y0 >= H) break;
        __syncthreads();
        for (int k = threadIdx.x; k < COUT * TS * TS; k += WG_THREADS) {
            const int co = k / (TS * TS), p = k % (TS * TS);
            const int yy = y0 + p / TS, xx = x0 + p % TS;
            gs[p * COUT + co] = (yy < H && xx < W) ? gb[co * HW + size_t(yy) * W + xx] : 0.0f;
        }
        for (int k = threadIdx.x; k < Cin * HALO * HALO; k += WG_THREADS) {
            const int c = k / (HALO * HALO), rr = k % (HALO * HALO);
            const int yy = y0 - 1 + rr / HALO, xx = x0 - 1 + rr % HALO;
            xs[k] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? inb[c * HW + size_t(yy) * W + xx] : 0.0f;
        }
        __syncthreads();
        if (gi < G) {
            const float* xc = xs + ci * HALO * HALO + (tap / 3) * HALO + tap % 3;
            for (int p = gi; p < TS * TS; p += G) {
                const float v = xc[(p / TS) * HALO + p % TS];
                const float* gp = gs + p * COUT;
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] = fmaf(gp[co], v, acc[co]);
            }
        }
        if (threadIdx.x < COUT)
            for (int p = 0; p < TS * TS; ++p) accb += gs[p * COUT + threadIdx.x];
    }
    __syncthreads();
    // sum the pixel groups: red[gi][co][q]
    float* red = sm;
    if (gi < G)
#pragma unroll
        for (int co = 0; co < COUT; ++co) red[(gi * COUT + co) * npairs + q] = acc[co];
    __syncthreads();
    const int nout = COUT * npairs;
    const size_t strip = (size_t(b) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float* part = partial + strip * (nout + COUT);
    for (int o = threadIdx.x; o < nout; o += WG_THREADS) {
        float s = 0.0f;
        for (int k = 0; k < G; ++k) s += red[k * nout + o];
        part[o] = s;                                  // o = co * Cin * 9 + ci * 9 + tap
    }
    if (threadIdx.x < COUT) part[nout + threadIdx.x] = accb;
}

// out[o] = sum_s partial[s][o] in strip order (deterministic)
__global__ void k_reduce_partials(const float* partial, int nstrips, int len, float* grad_w, float* grad_b,
                                  int nout) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < len; o += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < nstrips; ++k) s += partial[size_t(k) * len + o];
        if (o < nout) grad_w[o] = s;
        else grad_b[o - nout] = s;
    }
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* w, float* f, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        f[i] = __bfloat162float(w[i]);
}

__global__ void k_f32_to_bf16(const float* f, __nv_bfloat16* w, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        w[i] = __float2bfloat16_rn(f[i]);
}

// weights of the input-gradient correlation: w'[ci][co][tap] = w[co][ci][8 - tap]
__global__ void k_flip_weights(const __nv_bfloat16* w, float* wt, int Cin, int Cout) {
    const int n = Cin * Cout * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i / (Cout * 9), r = i % (Cout * 9), co = r / 9, k = r % 9;
        wt[i] = __bfloat162float(w[(co * Cin + ci) * 9 + (8 - k)]);
    }
}

// gradient through tanh: g *= 1 - a^2 (a = the layer's output)
__global__ void k_tanh_back(float* g, const float* a, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        g[i] *= 1.0f - a[i] * a[i];
}

// loss += mean (pred - target)^2; grad = 2 (pred - target) / n
__global__ void k_mse(const float* pred, const float* tgt, float* grad, float* loss, size_t n) {
    __shared__ float red[32];
    float s = 0.0f;
    const float sc = 2.0f / float(n);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float d = pred[i] - tgt[i];
        grad[i] = sc * d;
        s = fmaf(d, d, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < int(blockDim.x + 31) / 32; ++w) t += red[w];
        atomicAdd(loss, t / float(n));
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; the BF16 copy is the master rounded to nearest
__global__ void k_adam(float* master, __nv_bfloat16* wb, const float* grad, float* m, float* v, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = master[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        master[i] = w;
        if (wb) wb[i] = __float2bfloat16_rn(w);
    }
}

// ---- tensor-core forward (inference): implicit GEMM on mma.sync.m16n8k16 (bf16 in, FP32 accumulate).
// A CTA of 4 warps computes a 16 x 16 pixel tile; warp w owns output rows 4w .. 4w+3 (one m16 tile
// per row, rows of the m16 tile = the 16 pixels of that row), all NPAD output channels (NPAD/8 n8
// tiles).  GEMM: M = pixels, N = Cout, K = 9 Cin ordered k = tap * Cin + ci (padded to 16).  The
// input tile with its halo is staged as bf16 pairs [pixel][ci/2] and the weights as bf16 pairs
// [n][k/2]; the row strides are padded so that the fragment loads of a warp hit 32 distinct banks.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// IN_NHWC / OUT_NHWC: the layer input / output as bf16 [B][H][W][C] (the context's inference
// buffers between layers: what the next layer's staging would round to anyway) instead of FP32
// [B][C][H][W].  The results are the same either way.
template <int CIN, int NPAD, bool IN_NHWC, bool OUT_NHWC>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(const void* __restrict__ in_,
                                                    const __nv_bfloat16* __restrict__ w,
                                                    const float* __restrict__ bias, void* __restrict__ out_,
                                                    int Cout, int H, int W, int act) {
    constexpr int K = 9 * CIN;
    constexpr int KP = (K + 15) / 16 * 16;
    constexpr int KSW = KP / 2 + 4;                       // words per weight row
    constexpr int PSW = CIN / 2 + (CIN >= 32 ? 4 : 1);    // words per staged pixel
    constexpr int NT = NPAD / 8;
    __shared__ uint32_t ws[NPAD * KSW];
    __shared__ uint32_t xs[HALO * HALO * PSW];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TS, y0 = blockIdx.y * TS, b = blockIdx.z;
    const size_t HW = size_t(H) * W;
    for (int idx = tid; idx < NPAD * (KP / 2); idx += 128) {
        const int n = idx / (KP / 2), k0 = 2 * (idx % (KP / 2));
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = k0 + e;
            v[e] = (n < Cout && k < K) ? __bfloat162float(w[(n * CIN + k % CIN) * 9 + k / CIN]) : 0.0f;
        }
        ws[n * KSW + k0 / 2] = pack_bf16(v[0], v[1]);
    }
    if (IN_NHWC) {
        // CIN/2 words per pixel, copied 4 words (16 bytes) at a time when CIN is a multiple of 8
        const uint32_t* inb = reinterpret_cast<const uint32_t*>(in_) + size_t(b) * HW * (CIN / 2);
        constexpr int VW = (CIN % 8 == 0) ? 4 : 1;
        for (int idx = tid; idx < HALO * HALO * (CIN / 2 / VW); idx += 128) {
            const int p = idx / (CIN / 2 / VW), q = idx % (CIN / 2 / VW);
            const int yy = y0 - 1 + p / HALO, xx = x0 - 1 + p % HALO;
            const bool ok = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const size_t o = (size_t(yy) * W + xx) * (CIN / 2) + q * VW;
            if (VW == 4) {
                const uint4 v = ok ? *reinterpret_cast<const uint4*>(inb + o) : make_uint4(0u, 0u, 0u, 0u);
                uint32_t* d = xs + p * PSW + q * 4;
                d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
            } else {
                xs[p * PSW + q] = ok ? inb[o] : 0u;
            }
        }
    } else {
        const float* inb = reinterpret_cast<const float*>(in_) + size_t(b) * CIN * HW;
        for (int idx = tid; idx < HALO * HALO * (CIN / 2); idx += 128) {
            const int p = idx % (HALO * HALO), cw = idx / (HALO * HALO);
            const int yy = y0 - 1 + p / HALO, xx = x0 - 1 + p % HALO;
            float v0 = 0.0f, v1 = 0.0f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const size_t o = size_t(yy) * W + xx;
                v0 = inb[(2 * cw) * HW + o];
                v1 = inb[(2 * cw + 1) * HW + o];
            }
            xs[p * PSW + cw] = pack_bf16(v0, v1);
        }
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    float acc[4][NT][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll 2
    for (int s = 0; s < KP / 16; ++s) {
        uint32_t bf[NT][2];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int n = nt * 8 + g;
            bf[nt][0] = ws[n * KSW + s * 8 + t];
            bf[nt][1] = ws[n * KSW + s * 8 + 4 + t];
        }
        const int klo = s * 16 + 2 * t, khi = klo + 8;
        const bool vlo = klo < K, vhi = khi < K;
        const int tlo = klo / CIN, clo = (klo % CIN) / 2, thi = khi / CIN, chi = (khi % CIN) / 2;
        const int olo = (tlo / 3) * HALO + tlo % 3, ohi = (thi / 3) * HALO + thi % 3;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int row = (warp * 4 + mt) * HALO;           // output row of this m16 tile, box coordinates
            uint32_t af[4];
            af[0] = vlo ? xs[(row + olo + g) * PSW + clo] : 0u;
            af[1] = vlo ? xs[(row + olo + g + 8) * PSW + clo] : 0u;
            af[2] = vhi ? xs[(row + ohi + g) * PSW + chi] : 0u;
            af[3] = vhi ? xs[(row + ohi + g + 8) * PSW + chi] : 0u;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) mma_bf16_16816(acc[mt][nt], af, bf[nt]);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        const int y = y0 + warp * 4 + mt;
        if (y >= H) continue;
        if (OUT_NHWC) {
            // channel pairs (co, co + 1) as one bf16x2 word; Cout is even here
            uint32_t* ob = reinterpret_cast<uint32_t*>(out_) + size_t(b) * HW * (Cout / 2);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int x = x0 + g + hh * 8;
                    const int co = nt * 8 + 2 * t;
                    if (co < Cout && x < W) {
                        float v0 = acc[mt][nt][2 * hh] + bias[co], v1 = acc[mt][nt][2 * hh + 1] + bias[co + 1];
                        if (act) {
                            v0 = tanhf(v0);
                            v1 = tanhf(v1);
                        }
                        ob[(size_t(y) * W + x) * (Cout / 2) + co / 2] = pack_bf16(v0, v1);
                    }
                }
        } else {
            float* ob = reinterpret_cast<float*>(out_) + size_t(b) * Cout * HW;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int x = x0 + g + (e >= 2 ? 8 : 0);
                    const int co = nt * 8 + 2 * t + (e & 1);
                    if (co < Cout && x < W) {
                        const float v = acc[mt][nt][e] + bias[co];
                        ob[co * HW + size_t(y) * W + x] = act ? tanhf(v) : v;
                    }
                }
        }
    }
}

int grid_for(size_t n) {
    const size_t g = (n + 255) / 256;
    return int(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

size_t fwd_smem(int Cin, int Cout) { return sizeof(float) * (size_t(Cout) * Cin * 9 + size_t(Cin) * HALO * HALO); }
size_t wgrad_smem(int Cin, int Cout) {
    const size_t tile = sizeof(float) * (size_t(TS) * TS * Cout + size_t(Cin) * HALO * HALO);
    const size_t red = sizeof(float) * size_t(WG_THREADS) * Cout;   // G * npairs * COUT = 288 * COUT
    return tile > red ? tile : red;
}

template <int COUT>
cudaError_t fwd_launch(const float* in, const float* wf, const float* bias, float* out, int B, int Cin, int H, int W,
                       int act, cudaStream_t s) {
    dim3 grid((W + TS - 1) / TS, (H + TS - 1) / TS, B);
    k_conv_fwd<COUT><<<grid, TS * TS, fwd_smem(Cin, COUT), s>>>(in, wf, bias, out, Cin, H, W, act);
    return cudaGetLastError();
}

// strip height (tiles) so that the weight-gradient grid holds about 4 blocks per SM
int strip_rows(int B, int H, int W) {
    int nsm = 152;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long gx = (W + TS - 1) / TS, ty = (H + TS - 1) / TS;
    const long long want = 4LL * nsm;
    long long gy = (want + B * gx - 1) / (B * gx);
    if (gy < 1) gy = 1;
    if (gy > ty) gy = ty;
    return int((ty + gy - 1) / gy);
}

bool chan_ok(int c) { return c == 2 || c == 4 || c == 32; }

bool shape_ok(int B, int Cin, int Cout, int H, int W) {
    return B > 0 && H > 0 && W > 0 && chan_ok(Cin) && chan_ok(Cout) && (H + TS - 1) / TS <= 65535 &&
           B <= 65535 && (long long)B * MAXC * H * W < (1LL << 40);
}

}  // namespace

cudaError_t nn_prepare() {
    const int f32 = int(fwd_smem(MAXC, 32)), f4 = int(fwd_smem(MAXC, 4)), f2 = int(fwd_smem(MAXC, 2));
    cudaError_t e = cudaFuncSetAttribute(k_conv_fwd<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, f32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_fwd<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, f4);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_fwd<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, f2);
    const int g32 = int(wgrad_smem(MAXC, 32)), g4 = int(wgrad_smem(MAXC, 4)), g2 = int(wgrad_smem(MAXC, 2));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_wgrad<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, g32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_wgrad<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, g4);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_wgrad<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, g2);
    return e;
}

cudaError_t nn_bf16_to_float(const uint16_t* w, float* f, size_t n, cudaStream_t s) {
    k_bf16_to_f32<<<grid_for(n), 256, 0, s>>>((const __nv_bfloat16*)w, f, n);
    return cudaGetLastError();
}

template <bool IN_NHWC, bool OUT_NHWC>
cudaError_t conv_tc_launch(const void* in, const __nv_bfloat16* wb, const float* bias, void* out, int B, int Cin,
                           int Cout, int H, int W, int act, cudaStream_t s) {
    dim3 grid((W + TS - 1) / TS, (H + TS - 1) / TS, B);
#define ES_TC(CI, NP) k_conv_fwd_tc<CI, NP, IN_NHWC, OUT_NHWC><<<grid, 128, 0, s>>>(in, wb, bias, out, Cout, H, W, act)
    if (Cout <= 8) {
        switch (Cin) {
            case 2: ES_TC(2, 8); break;
            case 4: ES_TC(4, 8); break;
            case 32: ES_TC(32, 8); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (Cin) {
            case 2: ES_TC(2, 32); break;
            case 4: ES_TC(4, 32); break;
            case 32: ES_TC(32, 32); break;
            default: return cudaErrorInvalidValue;
        }
    }
#undef ES_TC
    return cudaGetLastError();
}

cudaError_t nn_conv_forward_bf16(const float* in, const uint16_t* w, const float* bias, float* out, int B, int Cin,
                                 int Cout, int H, int W, int act, cudaStream_t s) {
    return conv_tc_launch<false, false>(in, (const __nv_bfloat16*)w, bias, out, B, Cin, Cout, H, W, act, s);
}

cudaError_t nn_conv_forward_bf16_fmt(const void* in, bool in_nhwc, const uint16_t* w, const float* bias, void* out,
                                     bool out_nhwc, int B, int Cin, int Cout, int H, int W, int act, cudaStream_t s) {
    const __nv_bfloat16* wb = (const __nv_bfloat16*)w;
    if (out_nhwc && (Cout & 1)) return cudaErrorInvalidValue;
    if (in_nhwc)
        return out_nhwc ? conv_tc_launch<true, true>(in, wb, bias, out, B, Cin, Cout, H, W, act, s)
                        : conv_tc_launch<true, false>(in, wb, bias, out, B, Cin, Cout, H, W, act, s);
    return out_nhwc ? conv_tc_launch<false, true>(in, wb, bias, out, B, Cin, Cout, H, W, act, s)
                    : conv_tc_launch<false, false>(in, wb, bias, out, B, Cin, Cout, H, W, act, s);
}

cudaError_t nn_conv_forward_f32(const float* in, const float* wf, const float* bias, float* out, int B, int Cin,
                                int Cout, int H, int W, int act, cudaStream_t s) {
    switch (Cout) {
        case 2: return fwd_launch<2>(in, wf, bias, out, B, Cin, H, W, act, s);
        case 4: return fwd_launch<4>(in, wf, bias, out, B, Cin, H, W, act, s);
        case 32: return fwd_launch<32>(in, wf, bias, out, B, Cin, H, W, act, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace es

using namespace es;

extern "C" {

size_t es_nn_workspace_bytes(int B, int Cin, int Cout, int H, int W) {
    if (!shape_ok(B, Cin, Cout, H, W)) return 0;
    const int rows = strip_rows(B, H, W);
    const size_t gx = (W + TS - 1) / TS, gy = ((H + TS - 1) / TS + rows - 1) / rows;
    const size_t strips = size_t(B) * gx * gy;
    const size_t len = size_t(Cout) * Cin * 9 + Cout;
    return sizeof(float) * (size_t(Cout) * Cin * 9 + strips * len);
}

int es_nn_conv_forward(const float* in, const uint16_t* w, const float* bias, float* out, int B, int Cin, int Cout,
                       int H, int W, int act_tanh, void* workspace, size_t workspace_bytes, void* stream) {
    if (!in || !w || !out || !workspace || !shape_ok(B, Cin, Cout, H, W)) return ES_ERR_ARG;
    if (workspace_bytes < sizeof(float) * size_t(Cout) * Cin * 9) return ES_ERR_ARG;
    if (in == out) return ES_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* wf = (float*)workspace;
    if (nn_prepare() != cudaSuccess) return ES_ERR_CUDA;
    if (nn_bf16_to_float(w, wf, size_t(Cout) * Cin * 9, s) != cudaSuccess) return ES_ERR_CUDA;
    return nn_conv_forward_f32(in, wf, bias, out, B, Cin, Cout, H, W, act_tanh, s) == cudaSuccess ? ES_OK
                                                                                                : ES_ERR_CUDA;
}

int es_nn_conv_forward_bf16(const float* in, const uint16_t* w, const float* bias, float* out, int B, int Cin,
                            int Cout, int H, int W, int act_tanh, void* stream) {
    if (!in || !w || !bias || !out || !shape_ok(B, Cin, Cout, H, W) || in == out) return ES_ERR_ARG;
    return nn_conv_forward_bf16(in, w, bias, out, B, Cin, Cout, H, W, act_tanh, (cudaStream_t)stream) == cudaSuccess
               ? ES_OK
               : ES_ERR_CUDA;
}

int es_nn_conv_backward(const float* in, const uint16_t* w, const float* out, float* grad_out, float* grad_in,
                        float* grad_w, float* grad_b, int B, int Cin, int Cout, int H, int W, int act_tanh,
                        void* workspace, size_t workspace_bytes, void* stream) {
    if (!in || !w || !grad_out || !grad_w || !grad_b || !workspace || !shape_ok(B, Cin, Cout, H, W))
        return ES_ERR_ARG;
    if (act_tanh && !out) return ES_ERR_ARG;
    if (workspace_bytes < es_nn_workspace_bytes(B, Cin, Cout, H, W)) return ES_ERR_ARG;
    if (grad_in && (grad_in == grad_out || grad_in == in)) return ES_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (nn_prepare() != cudaSuccess) return ES_ERR_CUDA;
    const size_t nout_g = size_t(B) * Cout * H * W;
    if (act_tanh) k_tanh_back<<<grid_for(nout_g), 256, 0, s>>>(grad_out, out, nout_g);
    float* wt = (float*)workspace;
    float* partial = wt + size_t(Cout) * Cin * 9;
    const int rows = strip_rows(B, H, W);
    dim3 grid((W + TS - 1) / TS, ((H + TS - 1) / TS + rows - 1) / rows, B);
    const size_t sm = wgrad_smem(Cin, Cout);
    switch (Cout) {
        case 2: k_conv_wgrad<2><<<grid, WG_THREADS, sm, s>>>(in, grad_out, partial, Cin, H, W, rows); break;
        case 4: k_conv_wgrad<4><<<grid, WG_THREADS, sm, s>>>(in, grad_out, partial, Cin, H, W, rows); break;
        default: k_conv_wgrad<32><<<grid, WG_THREADS, sm, s>>>(in, grad_out, partial, Cin, H, W, rows); break;
    }
    const int nout = Cout * Cin * 9;
    const int strips = int(grid.x * grid.y * grid.z);
    k_reduce_partials<<<grid_for(size_t(nout + Cout)), 256, 0, s>>>(partial, strips, nout + Cout, grad_w, grad_b,
                                                                     nout);
    if (grad_in) {
        k_flip_weights<<<grid_for(size_t(nout)), 256, 0, s>>>((const __nv_bfloat16*)w, wt, Cin, Cout);
        if (nn_conv_forward_f32(grad_out, wt, nullptr, grad_in, B, Cout, Cin, H, W, 0, s) != cudaSuccess)
            return ES_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

int es_nn_to_bf16(const float* src, uint16_t* dst, int64_t n, void* stream) {
    if (!src || !dst || n <= 0) return ES_ERR_ARG;
    k_f32_to_bf16<<<grid_for(size_t(n)), 256, 0, (cudaStream_t)stream>>>(src, (__nv_bfloat16*)dst, size_t(n));
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

int es_nn_mse(const float* pred, const float* target, float* grad, float* loss, int64_t n, void* stream) {
    if (!pred || !target || !grad || !loss || n <= 0) return ES_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    k_mse<<<grid_for(size_t(n)), 256, 0, s>>>(pred, target, grad, loss, size_t(n));
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

int es_nn_adam(float* master, uint16_t* w_bf16, const float* grad, float* m, float* v, int n, float lr, float beta1,
               float beta2, float eps, int step, void* stream) {
    if (!master || !grad || !m || !v || n <= 0 || step < 1 || !(lr >= 0.0f)) return ES_ERR_ARG;
    const float c1 = float(1.0 / (1.0 - pow(double(beta1), double(step))));
    const float c2 = float(1.0 / (1.0 - pow(double(beta2), double(step))));
    k_adam<<<grid_for(size_t(n)), 256, 0, (cudaStream_t)stream>>>(master, (__nv_bfloat16*)w_bf16, grad, m, v, n, lr,
                                                                  beta1, beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

}  // extern "C"
