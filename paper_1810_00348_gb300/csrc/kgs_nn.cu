// kgs_nn.cu -- the 3D convolutional surrogate that supplies the initial
// macroscopic fields of a solve: inference and training kernels.
//
// Volumes are channels-last, act[b][z][y][x][Cp] with Cp the channel count
// padded to a multiple of 16; stored activations and weights are bfloat16,
// every product is accumulated in FP32.  A layer is a 3x3x3 convolution with
// zero padding, bias, and ReLU except on the last layer.  As a GEMM it is
// out[v][co] = sum_{t, ci} in[v + off(t)][ci] W[t][co][ci] (M = voxels,
// N = output channels, K = 27 * input channels).  The forward pass and the
// data gradient of the backward pass (the same GEMM with the taps mirrored and
// the channel roles swapped, ReLU-derivative mask in the epilogue) run on the
// tcgen05 tensor cores (kgs_conv_tc.cu).  This file holds
// the weight gradient (per tap a GEMM over voxels, M = Cout, N = Cin, K =
// voxels) also runs there, split over voxel chunks; this file adds its
// fixed-order reduction over chunks,
// plus bias gradients, the masked mean-squared-error loss, Adam, and the
// feature / target / prediction maps between the solver's FP64 fields and the
// network's normalised channels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/kgs.h"
#include "kgs_nn.h"

namespace {

using kgs::nn::ConvDims;

__host__ __device__ inline int pad16(int c) { return (c + 15) / 16 * 16; }

// gW[t][co][ci] = sum over (sample, chunk) in order of the partials.
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int n_parts, size_t per, float *__restrict__ gw)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per) return;
    float s = 0.f;
    for (int p = 0; p < n_parts; p++) s += part[(size_t)p * per + i];
    gw[i] = s;
}

// Bias gradient gb[co] = sum over voxels of dy[v][co]: one block per channel,
// strided per-thread sums then a tree (fixed order).
template <typename T>
__global__ void bias_grad_kernel(const T *__restrict__ dy, size_t nvox, int cp, float *__restrict__ gb)
{
    __shared__ float sh[256];
    const int co = blockIdx.x;
    float s = 0.f;
    for (size_t v = threadIdx.x; v < nvox; v += 256) s += (float)dy[v * cp + co];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[co] = sh[0];
}

// Wt[26-t][ci][co] = W[t][co][ci]: weights of the data-gradient convolution.
__global__ void transpose_w_kernel(const __nv_bfloat16 *__restrict__ w, int cout_p, int cin_p,
                                   __nv_bfloat16 *__restrict__ wt)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)cout_p * cin_p;
    if (i >= 27 * per) return;
    const int t = (int)(i / per), r = (int)(i % per), co = r / cin_p, ci = r % cin_p;
    wt[(size_t)(26 - t) * per + (size_t)ci * cout_p + co] = w[i];
}

// Masked mean squared error over the real output channels: per-block partial
// sums (fixed order) and the gradient dy = 2 (y - t) m / count as bf16.
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ tgt, const uint8_t *__restrict__ mask,
                           size_t nvox, int cp, int cout, float inv_count, __nv_bfloat16 *__restrict__ dy,
                           float *__restrict__ part)
{
    __shared__ float sh[256];
    float s = 0.f;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nvox) {
        const float mk = (mask == nullptr || mask[i]) ? 1.f : 0.f;
        for (int c = 0; c < cp; c++) {
            float g = 0.f;
            if (c < cout) {
                const float d = (y[i * cp + c] - tgt[i * cout + c]) * mk;
                s += d * d;
                g = 2.f * d * inv_count;
            }
            dy[i * cp + c] = __float2bfloat16_rn(g);
        }
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Adam on the FP32 master parameters (padding entries stay zero: their
// gradients are zero), and the bf16 copy used by the convolutions.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                            float *__restrict__ m2, __nv_bfloat16 *__restrict__ pb, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float pi = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float *__restrict__ x, size_t n, __nv_bfloat16 *__restrict__ y)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// Input channels-last FP32 [vox][c0] -> bf16 [vox][cp] (padding zero).
__global__ void pack_input_kernel(const float *__restrict__ x, size_t nvox, int c0, int cp,
                                  __nv_bfloat16 *__restrict__ y)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvox * cp) return;
    const size_t v = i / cp;
    const int c = (int)(i % cp);
    y[i] = __float2bfloat16_rn(c < c0 ? x[v * c0 + c] : 0.f);
}

// Output FP32 [vox][cp] -> [vox][cout].
__global__ void unpack_output_kernel(const float *__restrict__ y, size_t nvox, int cp, int cout, float *__restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvox * cout) return;
    out[i] = y[(i / cout) * cp + i % cout];
}

// ---------------------------------------------------------------------------
// Maps between the solver's macroscopic fields ([8][nz][ny][nx] FP64: rho,
// Ux, Uy, Uz, T, qx, qy, qz) and the network's normalised channels.  Each
// field c is scaled about its rest value: n_c = s_c (m_c - r_c) with
// r = (1, 0, 0, 0, 1, 0, 0, 0) and s = (10, 10, 10, 10, 50, 100, 100, 100),
// so that fields of a low-speed flow are O(1) in the network.
__constant__ float c_scale[8] = {10.f, 10.f, 10.f, 10.f, 50.f, 100.f, 100.f, 100.f};
__constant__ double c_rest[8] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0};

__device__ inline void up_axis(int i, int n, int nc, int &i0, int &i1, double &t)
{
    // cell centres of equal-width cells: fine centre (i + 1/2)/n lies at
    // coarse index (i + 1/2) nc / n - 1/2, clamped to the outermost centres
    double u = ((double)i + 0.5) * nc / n - 0.5;
    u = fmin(fmax(u, 0.0), (double)(nc - 1));
    i0 = (int)floor(u);
    i1 = min(i0 + 1, nc - 1);
    t = u - i0;
}

// Features of one instance: x[z][y][x][11] = (log Kn, 10 U_lid, solid,
// normalised upsampled coarse fields) and the upsampled fields themselves.
__global__ void features_kernel(int nx, int ny, int nz, int nxc, int nyc, int nzc, const double *__restrict__ coarse,
                                const uint8_t *__restrict__ solid, float log_kn, float u_lid, float *__restrict__ x,
                                double *__restrict__ up)
{
    const size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t ncell = (size_t)nx * ny * nz;
    if (cell >= ncell) return;
    const int i = (int)(cell % nx), j = (int)((cell / nx) % ny), k = (int)(cell / ((size_t)nx * ny));
    int i0, i1, j0, j1, k0, k1;
    double tx, ty, tz;
    up_axis(i, nx, nxc, i0, i1, tx);
    up_axis(j, ny, nyc, j0, j1, ty);
    up_axis(k, nz, nzc, k0, k1, tz);
    const size_t ncc = (size_t)nxc * nyc * nzc;
    float *xo = x + cell * 11;
    xo[0] = log_kn;
    xo[1] = 10.f * u_lid;
    xo[2] = solid ? (float)(solid[cell] != 0) : 0.f;
    for (int c = 0; c < 8; c++) {
        const double *f = coarse + c * ncc;
        auto at = [&](int kk, int jj, int ii) { return f[((size_t)kk * nyc + jj) * nxc + ii]; };
        const double v0 = (1 - tx) * at(k0, j0, i0) + tx * at(k0, j0, i1);
        const double v1 = (1 - tx) * at(k0, j1, i0) + tx * at(k0, j1, i1);
        const double v2 = (1 - tx) * at(k1, j0, i0) + tx * at(k1, j0, i1);
        const double v3 = (1 - tx) * at(k1, j1, i0) + tx * at(k1, j1, i1);
        const double v = (1 - tz) * ((1 - ty) * v0 + ty * v1) + tz * ((1 - ty) * v2 + ty * v3);
        up[c * ncell + cell] = v;
        xo[3 + c] = (float)(c_scale[c] * (v - c_rest[c]));
    }
}

// Training target: the normalised correction t[cell][c] = s_c (fine - up).
__global__ void target_kernel(size_t ncell, const double *__restrict__ fine, const double *__restrict__ up,
                              float *__restrict__ t)
{
    const size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    for (int c = 0; c < 8; c++) t[cell * 8 + c] = (float)(c_scale[c] * (fine[c * ncell + cell] - up[c * ncell + cell]));
}

// Initial guess m = up + y / s, and the count of cells where it is not a
// physical state (non-finite, rho <= 0 or T <= 0).
__global__ void apply_kernel(size_t ncell, const double *__restrict__ up, const float *__restrict__ y,
                             double *__restrict__ m, int *__restrict__ n_bad)
{
    const size_t cell = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    bool bad = false;
    for (int c = 0; c < 8; c++) {
        const double v = up[c * ncell + cell] + (double)y[cell * 8 + c] / c_scale[c];
        m[c * ncell + cell] = v;
        bad |= !isfinite(v);
        if (c == 0 || c == 4) bad |= !(v > 0.0);
    }
    if (bad) atomicAdd(n_bad, 1);
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }


cudaError_t run_conv(int mode, const __nv_bfloat16 *in, const __nv_bfloat16 *w, __nv_bfloat16 *wpk,
                     const float *bias, void *out, const __nv_bfloat16 *gate, ConvDims dm, int *err, cudaStream_t s)
{
    return kgs::nn::conv_tc(mode, in, w, wpk, bias, out, gate, dm, err, s);
}

}  // namespace

// ---------------------------------------------------------------------------
// network object

struct kgs_net {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int L = 0;
    std::vector<int> c, cp;             // real and padded channels per level (L + 1)
    std::vector<size_t> w_off, b_off;   // offsets into the flat parameter arrays
    size_t n_params = 0;                // padded parameter count
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // FP32 master, grad, Adam moments
    __nv_bfloat16 *pb = nullptr;        // bf16 copy of the parameters
    __nv_bfloat16 *wt = nullptr;        // transposed weights of one layer (data gradient)
    __nv_bfloat16 *wpk = nullptr;       // one layer's weights packed for the convolution kernel
    long long step = 0;
    // activation storage for the current shape
    int B = 0, D = 0, H = 0, W = 0;
    std::vector<__nv_bfloat16 *> act;   // L bf16 tensors: input, hidden outputs
    float *out = nullptr;               // last layer FP32 [vox][cp[L]]
    __nv_bfloat16 *ga = nullptr, *gb2 = nullptr;  // gradient ping-pong (bf16)
    float *wpart = nullptr;
    size_t wpart_cap = 0;
    float *loss_part = nullptr;
    size_t loss_part_cap = 0;
    float *h_loss = nullptr;
    int *d_err = nullptr;  // set by a convolution whose bounded wait gave up
    int *h_err = nullptr;  // pinned copy
};

namespace {

int err(cudaError_t e)
{
    if (e == cudaSuccess) return KGS_OK;
    if (e == cudaErrorMemoryAllocation) return KGS_ENOMEM;
    return KGS_ECUDA;
}

#define NN_CHECK(x)                        \
    do {                                   \
        cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) return err(e_); \
    } while (0)

void free_acts(kgs_net *n)
{
    for (auto *a : n->act) cudaFree(a);
    n->act.clear();
    if (n->out) cudaFree(n->out);
    if (n->ga) cudaFree(n->ga);
    if (n->gb2) cudaFree(n->gb2);
    n->out = nullptr;
    n->ga = n->gb2 = nullptr;
    n->B = n->D = n->H = n->W = 0;
}

int ensure_shape(kgs_net *n, int B, int D, int H, int W)
{
    if (n->B == B && n->D == D && n->H == H && n->W == W) return KGS_OK;
    free_acts(n);
    const size_t nvox = (size_t)B * D * H * W;
    int cmax = 0;
    for (int l = 0; l <= n->L; l++) cmax = std::max(cmax, n->cp[l]);
    n->act.assign(n->L, nullptr);
    for (int l = 0; l < n->L; l++) NN_CHECK(cudaMalloc(&n->act[l], nvox * n->cp[l] * sizeof(__nv_bfloat16)));
    NN_CHECK(cudaMalloc(&n->out, nvox * n->cp[n->L] * sizeof(float)));
    NN_CHECK(cudaMalloc(&n->ga, nvox * cmax * sizeof(__nv_bfloat16)));
    NN_CHECK(cudaMalloc(&n->gb2, nvox * cmax * sizeof(__nv_bfloat16)));
    n->B = B;
    n->D = D;
    n->H = H;
    n->W = W;
    return KGS_OK;
}

// Synchronise the network's stream and report a convolution whose bounded
// wait gave up (KGS_ETIMEOUT; the word is cleared for the next call).
int sync_and_check(kgs_net *n)
{
    NN_CHECK(cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NN_CHECK(cudaStreamSynchronize(n->stream));
    if (*n->h_err) {
        *n->h_err = 0;
        NN_CHECK(cudaMemset(n->d_err, 0, sizeof(int)));
        return KGS_ETIMEOUT;
    }
    return KGS_OK;
}

ConvDims dims(const kgs_net *n, int l) { return ConvDims{n->B, n->D, n->H, n->W, n->cp[l], n->cp[l + 1]}; }

int forward(kgs_net *n, const float *x)
{
    cudaStream_t s = n->stream;
    const size_t nvox = (size_t)n->B * n->D * n->H * n->W;
    pack_input_kernel<<<nblk(nvox * n->cp[0], 256), 256, 0, s>>>(x, nvox, n->c[0], n->cp[0], n->act[0]);
    NN_CHECK(cudaGetLastError());
    for (int l = 0; l < n->L; l++) {
        const __nv_bfloat16 *w = n->pb + n->w_off[l];
        const float *bias = n->p + n->b_off[l];
        if (l < n->L - 1)
            NN_CHECK(run_conv(0, n->act[l], w, n->wpk, bias, n->act[l + 1], nullptr, dims(n, l), n->d_err, s));
        else
            NN_CHECK(run_conv(1, n->act[l], w, n->wpk, bias, n->out, nullptr, dims(n, l), n->d_err, s));
    }
    return KGS_OK;
}

// Gradients of all parameters for the upstream gradient held in n->ga
// (bf16, [vox][cp[L]]), after forward().
int backward(kgs_net *n)
{
    cudaStream_t s = n->stream;
    const size_t nvox = (size_t)n->B * n->D * n->H * n->W;
    const int n_chunks = kgs::nn::wgrad_chunks(dims(n, 0));
    __nv_bfloat16 *gcur = n->ga, *gnext = n->gb2;
    for (int l = n->L - 1; l >= 0; l--) {
        const ConvDims dm = dims(n, l);
        const size_t per = (size_t)27 * dm.cout_p * dm.cin_p;
        // weight gradient
        const size_t need = (size_t)n->B * n_chunks * per;
        if (need > n->wpart_cap) {
            if (n->wpart) cudaFree(n->wpart);
            n->wpart = nullptr;
            NN_CHECK(cudaMalloc(&n->wpart, need * sizeof(float)));
            n->wpart_cap = need;
        }
        NN_CHECK(kgs::nn::wgrad_tc(n->act[l], gcur, n->wpart, dm, n->d_err, s));
        wgrad_reduce_kernel<<<nblk(per, 256), 256, 0, s>>>(n->wpart, n->B * n_chunks, per, n->g + n->w_off[l]);
        NN_CHECK(cudaGetLastError());
        bias_grad_kernel<__nv_bfloat16><<<dm.cout_p, 256, 0, s>>>(gcur, nvox, dm.cout_p, n->g + n->b_off[l]);
        NN_CHECK(cudaGetLastError());
        if (l == 0) break;
        // data gradient into layer l's input, masked by that layer's ReLU
        transpose_w_kernel<<<nblk(per, 256), 256, 0, s>>>(n->pb + n->w_off[l], dm.cout_p, dm.cin_p, n->wt);
        NN_CHECK(cudaGetLastError());
        const ConvDims db{n->B, n->D, n->H, n->W, dm.cout_p, dm.cin_p};
        NN_CHECK(run_conv(2, gcur, n->wt, n->wpk, nullptr, gnext, n->act[l], db, n->d_err, s));
        std::swap(gcur, gnext);
    }
    return KGS_OK;
}

}  // namespace

extern "C" {

int kgs_net_create(kgs_net **out, int n_layers, const int *channels, unsigned long long seed, void *stream)
{
    if (!out || n_layers < 1 || !channels) return KGS_EINVAL;
    for (int l = 0; l <= n_layers; l++)
        if (channels[l] < 1 || pad16(channels[l]) > 112) return KGS_EINVAL;
    kgs_net *n = new (std::nothrow) kgs_net();
    if (!n) return KGS_ENOMEM;
    cudaGetDevice(&n->dev);
    n->stream = static_cast<cudaStream_t>(stream);
    n->L = n_layers;
    for (int l = 0; l <= n_layers; l++) {
        n->c.push_back(channels[l]);
        n->cp.push_back(pad16(channels[l]));
    }
    size_t off = 0, wmax = 0;
    for (int l = 0; l < n_layers; l++) {
        n->w_off.push_back(off);
        const size_t per = (size_t)27 * n->cp[l + 1] * n->cp[l];
        wmax = std::max(wmax, per);
        off += per;
        n->b_off.push_back(off);
        off += n->cp[l + 1];
    }
    n->n_params = off;
    // He-normal initial weights over the real fan-in (Box-Muller on a
    // splitmix64 stream), zero biases and zero padding
    std::vector<float> h(off, 0.f);
    unsigned long long st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ULL;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < n_layers; l++) {
        const double sd = std::sqrt(2.0 / (27.0 * n->c[l])) * (l == n_layers - 1 ? 0.1 : 1.0);
        for (int t = 0; t < 27; t++)
            for (int co = 0; co < n->c[l + 1]; co++)
                for (int ci = 0; ci < n->c[l]; ci++) {
                    const double u1 = next(), u2 = next();
                    const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
                    h[n->w_off[l] + ((size_t)t * n->cp[l + 1] + co) * n->cp[l] + ci] = (float)(sd * z);
                }
    }
    auto fail = [&](int rc) {
        kgs_net_destroy(n);
        return rc;
    };
    if (cudaMalloc(&n->p, off * 4) != cudaSuccess || cudaMalloc(&n->g, off * 4) != cudaSuccess ||
        cudaMalloc(&n->m1, off * 4) != cudaSuccess || cudaMalloc(&n->m2, off * 4) != cudaSuccess ||
        cudaMalloc(&n->pb, off * 2) != cudaSuccess || cudaMalloc(&n->wt, wmax * 2) != cudaSuccess || cudaMalloc(&n->wpk, wmax * 2) != cudaSuccess ||
        cudaMallocHost(&n->h_loss, sizeof(float)) != cudaSuccess || cudaMalloc(&n->d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&n->h_err, sizeof(int)) != cudaSuccess)
        return fail(KGS_ENOMEM);
    if (cudaMemset(n->d_err, 0, sizeof(int)) != cudaSuccess) return fail(KGS_ECUDA);
    if (cudaMemcpy(n->p, h.data(), off * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->g, 0, off * 4) != cudaSuccess || cudaMemset(n->m1, 0, off * 4) != cudaSuccess ||
        cudaMemset(n->m2, 0, off * 4) != cudaSuccess)
        return fail(KGS_ECUDA);
    // those ran on the legacy default stream; n->stream may not wait for it
    if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) return fail(KGS_ECUDA);
    to_bf16_kernel<<<nblk(off, 256), 256, 0, n->stream>>>(n->p, off, n->pb);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(n->stream) != cudaSuccess) return fail(KGS_ECUDA);
    *out = n;
    return KGS_OK;
}

int kgs_net_num_params(kgs_net *n, long long *real, long long *padded)
{
    if (!n) return KGS_EINVAL;
    long long r = 0;
    for (int l = 0; l < n->L; l++) r += 27LL * n->c[l] * n->c[l + 1] + n->c[l + 1];
    if (real) *real = r;
    if (padded) *padded = (long long)n->n_params;
    return KGS_OK;
}

// Parameters in the unpadded layout: per layer W[27][cout][cin] then b[cout].
static void pack_unpadded(const kgs_net *n, const float *padded, float *flat)
{
    size_t k = 0;
    for (int l = 0; l < n->L; l++) {
        for (int t = 0; t < 27; t++)
            for (int co = 0; co < n->c[l + 1]; co++)
                for (int ci = 0; ci < n->c[l]; ci++)
                    flat[k++] = padded[n->w_off[l] + ((size_t)t * n->cp[l + 1] + co) * n->cp[l] + ci];
        for (int co = 0; co < n->c[l + 1]; co++) flat[k++] = padded[n->b_off[l] + co];
    }
}

static void unpack_unpadded(const kgs_net *n, const float *flat, float *padded)
{
    size_t k = 0;
    for (int l = 0; l < n->L; l++) {
        for (int t = 0; t < 27; t++)
            for (int co = 0; co < n->c[l + 1]; co++)
                for (int ci = 0; ci < n->c[l]; ci++)
                    padded[n->w_off[l] + ((size_t)t * n->cp[l + 1] + co) * n->cp[l] + ci] = flat[k++];
        for (int co = 0; co < n->c[l + 1]; co++) padded[n->b_off[l] + co] = flat[k++];
    }
}

int kgs_net_get(kgs_net *n, int what, float *host)
{
    if (!n || !host || what < 0 || what > 1) return KGS_EINVAL;
    std::vector<float> h(n->n_params);
    NN_CHECK(cudaStreamSynchronize(n->stream));
    NN_CHECK(cudaMemcpy(h.data(), what == 0 ? n->p : n->g, n->n_params * 4, cudaMemcpyDeviceToHost));
    pack_unpadded(n, h.data(), host);
    return KGS_OK;
}

int kgs_net_set_params(kgs_net *n, const float *host)
{
    if (!n || !host) return KGS_EINVAL;
    std::vector<float> h(n->n_params, 0.f);
    unpack_unpadded(n, host, h.data());
    NN_CHECK(cudaStreamSynchronize(n->stream));  // no kernel of the network still reads the parameters
    NN_CHECK(cudaMemcpy(n->p, h.data(), n->n_params * 4, cudaMemcpyHostToDevice));
    NN_CHECK(cudaMemset(n->m1, 0, n->n_params * 4));
    NN_CHECK(cudaMemset(n->m2, 0, n->n_params * 4));
    // the copy and the memsets ran on the legacy default stream; n->stream
    // may not wait for it
    NN_CHECK(cudaStreamSynchronize(cudaStreamLegacy));
    to_bf16_kernel<<<nblk(n->n_params, 256), 256, 0, n->stream>>>(n->p, n->n_params, n->pb);
    NN_CHECK(cudaGetLastError());
    n->step = 0;
    NN_CHECK(cudaStreamSynchronize(n->stream));
    return KGS_OK;
}

int kgs_net_forward(kgs_net *n, const float *x, int B, int D, int H, int W, float *y)
{
    if (!n || !x || !y || B < 1 || D < 1 || H < 1 || W < 1) return KGS_EINVAL;
    (void)cudaGetLastError();
    int rc;
    if ((rc = ensure_shape(n, B, D, H, W)) || (rc = forward(n, x))) return rc;
    const size_t nvox = (size_t)B * D * H * W;
    unpack_output_kernel<<<nblk(nvox * n->c[n->L], 256), 256, 0, n->stream>>>(n->out, nvox, n->cp[n->L],
                                                                              n->c[n->L], y);
    NN_CHECK(cudaGetLastError());
    return sync_and_check(n);
}

int kgs_net_train_step(kgs_net *n, const float *x, const float *target, const uint8_t *mask, int B, int D, int H,
                       int W, float lr, float *loss)
{
    if (!n || !x || !target || B < 1 || D < 1 || H < 1 || W < 1) return KGS_EINVAL;
    (void)cudaGetLastError();
    int rc;
    if ((rc = ensure_shape(n, B, D, H, W)) || (rc = forward(n, x))) return rc;
    const size_t nvox = (size_t)B * D * H * W;
    const unsigned nb = nblk(nvox, 256);
    if (nb > n->loss_part_cap) {
        if (n->loss_part) cudaFree(n->loss_part);
        n->loss_part = nullptr;
        NN_CHECK(cudaMalloc(&n->loss_part, nb * sizeof(float)));
        n->loss_part_cap = nb;
    }
    // masked voxel count on the host is not needed: the mask is a device
    // array; count = voxels x channels when no mask is given, else the caller
    // passes a mask whose count the loss normalises over (see below)
    float count = (float)nvox;
    if (mask) {
        std::vector<uint8_t> hm(nvox);
        NN_CHECK(cudaMemcpyAsync(hm.data(), mask, nvox, cudaMemcpyDeviceToHost, n->stream));
        NN_CHECK(cudaStreamSynchronize(n->stream));
        size_t k = 0;
        for (uint8_t v : hm) k += v != 0;
        count = (float)std::max<size_t>(k, 1);
    }
    const int cL = n->c[n->L], cpL = n->cp[n->L];
    mse_kernel<<<nb, 256, 0, n->stream>>>(n->out, target, mask, nvox, cpL, cL, 1.f / (count * cL), n->ga,
                                          n->loss_part);
    NN_CHECK(cudaGetLastError());
    if ((rc = backward(n)) || (rc = sync_and_check(n))) return rc;  // no update from an incomplete pass
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    if (lr > 0.f) {
        adam_kernel<<<nblk(n->n_params, 256), 256, 0, n->stream>>>(n->p, n->g, n->m1, n->m2, n->pb, n->n_params, lr,
                                                                   b1, b2, 1e-8f, c1, c2);
        NN_CHECK(cudaGetLastError());
    }
    if (loss) {
        std::vector<float> hp(nb);
        NN_CHECK(cudaMemcpyAsync(hp.data(), n->loss_part, nb * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
        NN_CHECK(cudaStreamSynchronize(n->stream));
        double s = 0.0;
        for (float v : hp) s += v;
        *loss = (float)(s / (count * cL));
    }
    return KGS_OK;
}

int kgs_surrogate_features(int nx, int ny, int nz, int nxc, int nyc, int nzc, const double *coarse,
                           const uint8_t *solid, double kn, double u_lid, float *x, double *up, void *stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || nxc < 1 || nyc < 1 || nzc < 1 || !coarse || !x || !up || !(kn > 0.0))
        return KGS_EINVAL;
    const size_t ncell = (size_t)nx * ny * nz;
    features_kernel<<<nblk(ncell, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        nx, ny, nz, nxc, nyc, nzc, coarse, solid, (float)std::log(kn), (float)u_lid, x, up);
    NN_CHECK(cudaGetLastError());
    return KGS_OK;
}

int kgs_surrogate_target(long long ncell, const double *fine, const double *up, float *target, void *stream)
{
    if (ncell < 1 || !fine || !up || !target) return KGS_EINVAL;
    target_kernel<<<nblk((size_t)ncell, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>((size_t)ncell, fine, up,
                                                                                           target);
    NN_CHECK(cudaGetLastError());
    return KGS_OK;
}

int kgs_surrogate_apply(long long ncell, const double *up, const float *y, double *macros, int *n_bad, void *stream)
{
    if (ncell < 1 || !up || !y || !macros || !n_bad) return KGS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *d_bad = nullptr;
    NN_CHECK(cudaMallocAsync(reinterpret_cast<void **>(&d_bad), sizeof(int), st));
    cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        apply_kernel<<<nblk((size_t)ncell, 256), 256, 0, st>>>((size_t)ncell, up, y, macros, d_bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(n_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_bad, st);
    return err(e);
}

void kgs_net_destroy(kgs_net *n)
{
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    free_acts(n);
    float *bufs[] = {n->p, n->g, n->m1, n->m2, n->wpart, n->loss_part};
    for (float *b : bufs)
        if (b) cudaFree(b);
    if (n->pb) cudaFree(n->pb);
    if (n->wt) cudaFree(n->wt);
    if (n->wpk) cudaFree(n->wpk);
    if (n->h_loss) cudaFreeHost(n->h_loss);
    if (n->d_err) cudaFree(n->d_err);
    if (n->h_err) cudaFreeHost(n->h_err);
    delete n;
}

}  // extern "C"
