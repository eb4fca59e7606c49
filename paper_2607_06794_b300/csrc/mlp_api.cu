// Small multilayer perceptron used to propose sweep points from deposit
// descriptors: x[n_in] -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3.
// Loss L = 1/(2B) sum_b sum_k (y_bk - t_bk)^2.  Forward, backward and Adam are
// single-block kernels (a few thousand parameters and a few hundred samples:
// far too small for tensor cores to matter).  FP32 for training, FP64 for
// checking gradients.  The paper has no counterpart; it is the learned part of
// the batched parameter sweep.
#include <math.h>

#include <algorithm>

#include "../../include/lbm.h"

namespace {

constexpr int MLP_THREADS = 256;
constexpr int MAX_HIDDEN = 256;
constexpr int MAX_IO = 16;

template <typename T>
struct Net {
    const T* W1;
    const T* b1;
    const T* W2;
    const T* b2;
    const T* W3;
    const T* b3;
};

template <typename T>
__device__ Net<T> unpack(const T* p, int I, int H, int O) {
    Net<T> n;
    n.W1 = p;
    n.b1 = n.W1 + H * I;
    n.W2 = n.b1 + H;
    n.b2 = n.W2 + H * H;
    n.W3 = n.b2 + H;
    n.b3 = n.W3 + O * H;
    return n;
}

template <typename T>
__device__ T tanh_t(T v);
template <>
__device__ float tanh_t<float>(float v) { return tanhf(v); }
template <>
__device__ double tanh_t<double>(double v) { return tanh(v); }

// Forward pass of sample rows [b0, b1) of the batch; activations kept in a1/a2
// ([B][H]) when they are non-null.
template <typename T>
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_forward(const T* __restrict__ prm, int I, int H, int O, const T* __restrict__ x, int B,
                  T* __restrict__ y, T* __restrict__ a1, T* __restrict__ a2) {
    const Net<T> n = unpack(prm, I, H, O);
    __shared__ T h1[MAX_HIDDEN], h2[MAX_HIDDEN], xin[MAX_IO];
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < I) xin[threadIdx.x] = x[b * I + threadIdx.x];
        __syncthreads();
        for (int j = threadIdx.x; j < H; j += blockDim.x) {
            T s = n.b1[j];
            for (int k = 0; k < I; ++k) s += n.W1[j * I + k] * xin[k];
            h1[j] = tanh_t(s);
            if (a1) a1[b * H + j] = h1[j];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < H; j += blockDim.x) {
            T s = n.b2[j];
            for (int k = 0; k < H; ++k) s += n.W2[j * H + k] * h1[k];
            h2[j] = tanh_t(s);
            if (a2) a2[b * H + j] = h2[j];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < O; j += blockDim.x) {
            T s = n.b3[j];
            for (int k = 0; k < H; ++k) s += n.W3[j * H + k] * h2[k];
            y[b * O + j] = s;
        }
    }
}

// Backward pass over the whole batch in one block: gradient of L with respect
// to every parameter, summed over samples in a fixed order (deterministic).
template <typename T>
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_backward(const T* __restrict__ prm, int I, int H, int O, const T* __restrict__ x,
                   const T* __restrict__ t, int B, const T* __restrict__ y, const T* __restrict__ a1,
                   const T* __restrict__ a2, T* __restrict__ grad, T* __restrict__ loss,
                   T* __restrict__ d2buf, T* __restrict__ d1buf) {
    const Net<T> n = unpack(prm, I, H, O);
    const int P = H * I + H + H * H + H + O * H + O;
    T* gW1 = grad;
    T* gb1 = gW1 + H * I;
    T* gW2 = gb1 + H;
    T* gb2 = gW2 + H * H;
    T* gW3 = gb2 + H;
    T* gb3 = gW3 + O * H;
    const T invB = T(1) / T(B);
    // output error e = (y - t)/B and the two hidden deltas per sample
    __shared__ T red[MLP_THREADS];
    T l = 0;
    for (int q = threadIdx.x; q < B * O; q += blockDim.x) {
        const T e = y[q] - t[q];
        l += e * e;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = T(0.5) * red[0] * invB;
    // delta2[b][j] = (sum_k W3[k][j] e[b][k]) (1 - a2^2)
    for (int q = threadIdx.x; q < B * H; q += blockDim.x) {
        const int b = q / H, j = q % H;
        T s = 0;
        for (int k = 0; k < O; ++k) s += n.W3[k * H + j] * (y[b * O + k] - t[b * O + k]) * invB;
        const T a = a2[q];
        d2buf[q] = s * (T(1) - a * a);
    }
    __syncthreads();
    // delta1[b][j] = (sum_k W2[k][j] delta2[b][k]) (1 - a1^2)
    for (int q = threadIdx.x; q < B * H; q += blockDim.x) {
        const int b = q / H, j = q % H;
        T s = 0;
        for (int k = 0; k < H; ++k) s += n.W2[k * H + j] * d2buf[b * H + k];
        const T a = a1[q];
        d1buf[q] = s * (T(1) - a * a);
    }
    __syncthreads();
    // parameter gradients: one thread per parameter, batch summed in order
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        T g = 0;
        if (p < H * I) {
            const int j = p / I, k = p % I;
            for (int b = 0; b < B; ++b) g += d1buf[b * H + j] * x[b * I + k];
            gW1[p] = g;
        } else if (p < H * I + H) {
            const int j = p - H * I;
            for (int b = 0; b < B; ++b) g += d1buf[b * H + j];
            gb1[j] = g;
        } else if (p < H * I + H + H * H) {
            const int q = p - (H * I + H), j = q / H, k = q % H;
            for (int b = 0; b < B; ++b) g += d2buf[b * H + j] * a1[b * H + k];
            gW2[q] = g;
        } else if (p < H * I + 2 * H + H * H) {
            const int j = p - (H * I + H + H * H);
            for (int b = 0; b < B; ++b) g += d2buf[b * H + j];
            gb2[j] = g;
        } else if (p < H * I + 2 * H + H * H + O * H) {
            const int q = p - (H * I + 2 * H + H * H), k = q / H, j = q % H;
            for (int b = 0; b < B; ++b) g += (y[b * O + k] - t[b * O + k]) * invB * a2[b * H + j];
            gW3[q] = g;
        } else {
            const int k = p - (H * I + 2 * H + H * H + O * H);
            for (int b = 0; b < B; ++b) g += (y[b * O + k] - t[b * O + k]) * invB;
            gb3[k] = g;
        }
    }
}

// Adam with bias correction (step count t >= 1)
template <typename T>
__global__ void k_mlp_adam(T* __restrict__ prm, const T* __restrict__ g, T* __restrict__ m, T* __restrict__ v,
                           int P, T lr, T b1, T b2, T eps, int t) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const T mm = b1 * m[p] + (T(1) - b1) * g[p];
    const T vv = b2 * v[p] + (T(1) - b2) * g[p] * g[p];
    m[p] = mm;
    v[p] = vv;
    const T mh = mm / (T(1) - pow(b1, (T)t));
    const T vh = vv / (T(1) - pow(b2, (T)t));
    prm[p] -= lr * mh / (sqrt(vh) + eps);
}

bool dims_ok(int I, int H, int O, int B) {
    return I >= 1 && I <= MAX_IO && O >= 1 && O <= MAX_IO && H >= 1 && H <= MAX_HIDDEN && B >= 1;
}

template <typename T>
lbm_status forward(const void* prm, int I, int H, int O, const void* x, int B, void* y, void* act,
                   cudaStream_t st) {
    T* a1 = act ? (T*)act : nullptr;
    T* a2 = act ? (T*)act + (size_t)B * H : nullptr;
    k_mlp_forward<T><<<std::min(B, 1024), MLP_THREADS, 0, st>>>((const T*)prm, I, H, O, (const T*)x, B,
                                                                 (T*)y, a1, a2);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

template <typename T>
lbm_status loss_grad(const void* prm, int I, int H, int O, const void* x, const void* t, int B, void* y,
                     void* grad, void* loss, void* scratch, cudaStream_t st) {
    T* a1 = (T*)scratch;
    T* a2 = a1 + (size_t)B * H;
    T* d2 = a2 + (size_t)B * H;
    T* d1 = d2 + (size_t)B * H;
    lbm_status s = forward<T>(prm, I, H, O, x, B, y, a1, st);
    if (s != LBM_OK) return s;
    k_mlp_backward<T><<<1, MLP_THREADS, 0, st>>>((const T*)prm, I, H, O, (const T*)x, (const T*)t, B,
                                                  (const T*)y, a1, a2, (T*)grad, (T*)loss, d2, d1);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // namespace

extern "C" {

size_t lbm_mlp_param_count(int n_in, int n_hidden, int n_out) {
    if (!dims_ok(n_in, n_hidden, n_out, 1)) return 0;
    return (size_t)n_hidden * n_in + n_hidden + (size_t)n_hidden * n_hidden + n_hidden +
           (size_t)n_out * n_hidden + n_out;
}

size_t lbm_mlp_scratch_bytes(int dtype, int n_hidden, int batch) {
    return (size_t)4 * n_hidden * batch * (dtype == 1 ? 8 : 4);
}

lbm_status lbm_mlp_forward(int dtype, const void* params, int n_in, int n_hidden, int n_out, const void* x,
                           int batch, void* y, void* stream) {
    if (!params || !x || !y || !dims_ok(n_in, n_hidden, n_out, batch) || (dtype != 0 && dtype != 1))
        return LBM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == 0 ? forward<float>(params, n_in, n_hidden, n_out, x, batch, y, nullptr, st)
                      : forward<double>(params, n_in, n_hidden, n_out, x, batch, y, nullptr, st);
}

lbm_status lbm_mlp_loss_grad(int dtype, const void* params, int n_in, int n_hidden, int n_out, const void* x,
                             const void* targets, int batch, void* y, void* grad, void* loss, void* scratch,
                             size_t scratch_bytes, void* stream) {
    if (!params || !x || !targets || !y || !grad || !scratch || !dims_ok(n_in, n_hidden, n_out, batch) ||
        (dtype != 0 && dtype != 1))
        return LBM_EINVAL;
    if (scratch_bytes < lbm_mlp_scratch_bytes(dtype, n_hidden, batch)) return LBM_ENOMEM_WS;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == 0 ? loss_grad<float>(params, n_in, n_hidden, n_out, x, targets, batch, y, grad, loss,
                                         scratch, st)
                      : loss_grad<double>(params, n_in, n_hidden, n_out, x, targets, batch, y, grad, loss,
                                          scratch, st);
}

lbm_status lbm_mlp_adam(int dtype, void* params, const void* grad, void* m, void* v, int n_params, double lr,
                        double beta1, double beta2, double eps, int step, void* stream) {
    if (!params || !grad || !m || !v || n_params < 1 || step < 1 || (dtype != 0 && dtype != 1))
        return LBM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const int bt = 256, nb = (n_params + bt - 1) / bt;
    if (dtype == 0)
        k_mlp_adam<float><<<nb, bt, 0, st>>>((float*)params, (const float*)grad, (float*)m, (float*)v, n_params,
                                             (float)lr, (float)beta1, (float)beta2, (float)eps, step);
    else
        k_mlp_adam<double><<<nb, bt, 0, st>>>((double*)params, (const double*)grad, (double*)m, (double*)v,
                                              n_params, lr, beta1, beta2, eps, step);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

}  // extern "C"
