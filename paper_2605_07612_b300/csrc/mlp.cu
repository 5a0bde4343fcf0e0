// C ABI of the learned refinement-flag predictor (kernels in mlp.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/amr.h"
#include "mlp.cuh"
#include "mlp_tc.cuh"

using namespace amrb;

namespace {

#define MCU(call)                                                  \
    do {                                                           \
        if ((call) != cudaSuccess) {                               \
            cudaGetLastError();                                    \
            return AMR_ECUDA;                                      \
        }                                                          \
    } while (0)

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &s) { return double(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

size_t grad_smem(int F) {
    const MlpLayout L(F);
    return sizeof(float) * (size_t((L.n + 3) & ~int64_t(3)) + size_t(F) * kMlpTile + 4 * size_t(kMlpTile) * kMlpH +
                            size_t(kMlpTile) * kMlpO);
}

amr_status ensure_idx(amr_mlp *m, int64_t n) {
    if (m->idx_cap >= n) return AMR_OK;
    cudaFree(m->idx);
    m->idx = nullptr;
    m->idx_cap = 0;
    MCU(cudaMalloc(&m->idx, sizeof(int32_t) * size_t(std::max<int64_t>(n, 1))));
    m->idx_cap = n;
    return AMR_OK;
}

constexpr int kGradRows = 148;   // CTAs of one gradient launch (rows of `partial`)

// one gradient of the mean loss over samples idx[0..nb) into m->grad (P
// entries, then the loss)
amr_status gradient(amr_mlp *m, const float *x, int64_t n_total, const int32_t *idx, const int8_t *y, int64_t nb, cudaStream_t st) {
    const int64_t n1 = m->P + 1;
    const int rows = int(std::min<int64_t>(kGradRows, (nb + kMlpTile - 1) / kMlpTile));
    MCU(cudaMemsetAsync(m->partial, 0, sizeof(float) * size_t(n1) * size_t(rows), st));
    if (m->precision == 16)
        k_mlp_grad_tc<<<rows, 128, TcGradSmem(m->F).end, st>>>(m->wb, m->F, x, n_total, idx, y, nb, m->partial);
    else
        k_mlp_grad<<<rows, 128, grad_smem(m->F), st>>>(m->wb, m->F, x, n_total, idx, y, nb, m->partial);
    k_mlp_reduce<<<int((n1 + 255) / 256), 256, 0, st>>>(m->partial, rows, n1, m->grad);
    MCU(cudaGetLastError());
    return AMR_OK;
}

}  // namespace

extern "C" {

amr_status amr_mlp_create(int n_features, uint64_t seed, amr_mlp **out) {
    if (!out || n_features < 1 || n_features > kMlpMaxF) return AMR_EINVAL;
    *out = nullptr;
    amr_mlp *m = new (std::nothrow) amr_mlp();
    if (!m) return AMR_ENOMEM;
    m->F = n_features;
    m->P = MlpLayout(n_features).n;
    const size_t pb = sizeof(float) * size_t(m->P);
    bool ok = cudaMalloc(&m->w, pb) == cudaSuccess && cudaMalloc(&m->m, pb) == cudaSuccess &&
              cudaMalloc(&m->v, pb) == cudaSuccess && cudaMalloc(&m->grad, pb + sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * size_t(m->P)) == cudaSuccess &&
              cudaMalloc(&m->partial, (pb + sizeof(float)) * kGradRows) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(grad_smem(n_features))) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(pb)) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TcSmem(n_features).end)) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mlp_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TcGradSmem(n_features).end)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        amr_mlp_destroy(m);
        return AMR_ECUDA;
    }
    // uniform initialisation in +-1/sqrt(fan_in) (a published default for
    // ReLU-like layers), zero biases
    const MlpLayout L(n_features);
    std::vector<float> w(size_t(m->P), 0.f);
    uint64_t s = seed;
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        const double a = 1.0 / std::sqrt(double(fan_in));
        for (int64_t i = 0; i < count; ++i) w[size_t(off + i)] = float((2.0 * uniform01(s) - 1.0) * a);
    };
    fill(L.w1, int64_t(n_features) * kMlpH, n_features);
    fill(L.w2, kMlpH * kMlpH, kMlpH);
    fill(L.w3, kMlpH * kMlpO, kMlpH);
    amr_status r = amr_mlp_set_params(m, w.data(), m->P);
    if (r != AMR_OK) {
        amr_mlp_destroy(m);
        return r;
    }
    *out = m;
    return AMR_OK;
}

amr_status amr_mlp_destroy(amr_mlp *m) {
    if (!m) return AMR_OK;
    cudaFree(m->w);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->wb);
    cudaFree(m->partial);
    cudaFree(m->idx);
    delete m;
    return AMR_OK;
}

amr_status amr_mlp_n_params(const amr_mlp *m, int64_t *n) {
    if (!m || !n) return AMR_EINVAL;
    *n = m->P;
    return AMR_OK;
}

amr_status amr_mlp_get_params(const amr_mlp *m, float *host, int64_t n) {
    if (!m || !host || n != m->P) return AMR_EINVAL;
    MCU(cudaMemcpy(host, m->w, sizeof(float) * size_t(n), cudaMemcpyDeviceToHost));
    return AMR_OK;
}

amr_status amr_mlp_set_params(amr_mlp *m, const float *host, int64_t n) {
    if (!m || !host || n != m->P) return AMR_EINVAL;
    const size_t pb = sizeof(float) * size_t(n);
    MCU(cudaMemcpy(m->w, host, pb, cudaMemcpyHostToDevice));
    MCU(cudaMemset(m->m, 0, pb));
    MCU(cudaMemset(m->v, 0, pb));
    m->step = 0;
    k_to_bf16<<<int((n + 255) / 256), 256>>>(m->w, m->wb, n);
    MCU(cudaGetLastError());
    MCU(cudaDeviceSynchronize());
    return AMR_OK;
}

amr_status amr_mlp_set_precision(amr_mlp *m, int bits) {
    if (!m || (bits != 16 && bits != 32)) return AMR_EINVAL;
    m->precision = bits;
    return AMR_OK;
}

amr_status amr_mlp_forward(amr_mlp *m, const float *x, int64_t n, float *prob, amr_stream stream) {
    if (!m || (n > 0 && (!x || !prob)) || n < 0) return AMR_EINVAL;
    if (n == 0) return AMR_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (m->precision == 16) {
        const int grid = int(std::min<int64_t>((n + kTcTile - 1) / kTcTile, 2 * 148));
        k_mlp_forward_tc<<<grid, 128, TcSmem(m->F).end, st>>>(m->wb, m->F, x, n, prob);
    } else {
        const int grid = int(std::min<int64_t>((n + 127) / 128, 4 * 148));
        k_mlp_forward<<<grid, 128, sizeof(float) * size_t(m->P), st>>>(m->wb, m->F, x, n, prob);
    }
    MCU(cudaGetLastError());
    return AMR_OK;
}

amr_status amr_mlp_gradient(amr_mlp *m, const float *x, const int8_t *y, int64_t n, float *grad, amr_stream stream) {
    if (!m || !x || !y || !grad || n < 1) return AMR_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    amr_status r = ensure_idx(m, n);
    if (r != AMR_OK) return r;
    std::vector<int32_t> id(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) id[size_t(i)] = int32_t(i);
    MCU(cudaMemcpyAsync(m->idx, id.data(), sizeof(int32_t) * size_t(n), cudaMemcpyHostToDevice, st));
    if ((r = gradient(m, x, n, m->idx, y, n, st)) != AMR_OK) return r;
    MCU(cudaMemcpyAsync(grad, m->grad, sizeof(float) * size_t(m->P + 1), cudaMemcpyDeviceToDevice, st));
    MCU(cudaStreamSynchronize(st));
    return AMR_OK;
}

amr_status amr_mlp_adamw_step(amr_mlp *m, const float *grad, double lr, double weight_decay, amr_stream stream) {
    if (!m || !grad) return AMR_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    ++m->step;
    const float c1 = float(1.0 - std::pow(double(b1), double(m->step)));
    const float c2 = float(1.0 - std::pow(double(b2), double(m->step)));
    k_adamw<<<int((m->P + 255) / 256), 256, 0, st>>>(m->w, m->m, m->v, m->wb, grad, m->P, float(lr), b1, b2, eps,
                                                    float(weight_decay), c1, c2);
    MCU(cudaGetLastError());
    return AMR_OK;
}

amr_status amr_mlp_train(amr_mlp *m, const float *x, const int8_t *y, int64_t n, int epochs, int batch, double lr,
                         double weight_decay, uint64_t seed, double *final_loss, amr_stream stream) {
    if (!m || !x || !y || n < 1 || epochs < 1 || batch < 1) return AMR_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    amr_status r = ensure_idx(m, n);
    if (r != AMR_OK) return r;
    std::vector<int32_t> perm(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) perm[size_t(i)] = int32_t(i);
    uint64_t s = seed;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t i = n - 1; i > 0; --i) std::swap(perm[size_t(i)], perm[size_t(splitmix(s) % uint64_t(i + 1))]);
        MCU(cudaMemcpyAsync(m->idx, perm.data(), sizeof(int32_t) * size_t(n), cudaMemcpyHostToDevice, st));
        double sum = 0.0;
        int nbatch = 0;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - b0);
            if ((r = gradient(m, x, n, m->idx + b0, y, nb, st)) != AMR_OK) return r;
            ++m->step;
            const float c1 = float(1.0 - std::pow(double(b1), double(m->step)));
            const float c2 = float(1.0 - std::pow(double(b2), double(m->step)));
            k_adamw<<<int((m->P + 255) / 256), 256, 0, st>>>(m->w, m->m, m->v, m->wb, m->grad, m->P, float(lr), b1, b2, eps,
                                                            float(weight_decay), c1, c2);
            MCU(cudaGetLastError());
            if (e == epochs - 1) {
                float l = 0.f;
                MCU(cudaMemcpyAsync(&l, m->grad + m->P, sizeof(float), cudaMemcpyDeviceToHost, st));
                MCU(cudaStreamSynchronize(st));
                sum += l;
                ++nbatch;
            }
        }
        last = nbatch ? sum / nbatch : 0.0;
    }
    MCU(cudaStreamSynchronize(st));
    if (final_loss) *final_loss = last;
    return AMR_OK;
}

}  // extern "C"
