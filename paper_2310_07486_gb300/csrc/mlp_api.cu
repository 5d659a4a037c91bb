// mlp_api.cu -- host side of the learned-ladder MLP entry points of qsg.h:
// workspace carving, uploads, and the ordering of training launches.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "qsg.h"
#include "qsg_launch.h"

using namespace qsg;

namespace {

constexpr size_t kAlignM = 256;
constexpr int kChunk = 256;  // training steps per index upload
constexpr int kMaxBatch = 4096;

size_t up(size_t v) { return (v + kAlignM - 1) / kAlignM * kAlignM; }

struct Layout {
    float *P, *M, *V, *grad, *partial, *lossp, *losses, *X, *T, *Xp, *Yp;
    __nv_bfloat16 *Pb;
    int *idx;
};

size_t carve_mlp(char *base, long long n_data, int max_batch, Layout *l) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off = up(off + bytes);
        return p;
    };
    const size_t np = (size_t)mlp_param_count();
    const size_t tiles = (size_t)(max_batch + 15) / 16;
    Layout t;
    t.P = (float *)take(np * 4);
    t.M = (float *)take(np * 4);
    t.V = (float *)take(np * 4);
    t.grad = (float *)take(np * 4);
    t.Pb = (__nv_bfloat16 *)take(np * 2);
    t.partial = (float *)take(tiles * np * 4);
    t.lossp = (float *)take(tiles * 4);
    t.losses = (float *)take((size_t)kChunk * 4);
    t.idx = (int *)take((size_t)kChunk * max_batch * 4);
    t.X = (float *)take((size_t)n_data * 64 * 4);
    t.T = (float *)take((size_t)n_data * 33 * 4);
    t.Xp = (float *)take((size_t)n_data * 64 * 4);
    t.Yp = (float *)take((size_t)n_data * 33 * 4);
    if (l) *l = t;
    return off;
}

}  // namespace

struct qsg_mlp {
    Layout l;
    long long n_data = 0, n_loaded = 0;
    int max_batch = 0;
    int step = 0;  // Adam steps taken since the parameters were set
    cudaStream_t st = nullptr;
    bool has_params = false;
};

#define MLP_CUDA(expr)                                \
    do {                                              \
        if ((expr) != cudaSuccess) return QSG_ERR_CUDA; \
    } while (0)

extern "C" {

int32_t qsg_mlp_param_count(void) { return (int32_t)mlp_param_count(); }

size_t qsg_mlp_workspace_bytes(int64_t n_data, int32_t max_batch) {
    if (n_data < 1 || max_batch < 1 || max_batch > kMaxBatch) return 0;
    return carve_mlp(nullptr, n_data, max_batch, nullptr);
}

qsg_status qsg_mlp_create(qsg_mlp **out, void *d_workspace, size_t workspace_bytes, int64_t n_data,
                          int32_t max_batch, void *cuda_stream) {
    if (!out) return QSG_ERR_ARG;
    *out = nullptr;
    const size_t need = qsg_mlp_workspace_bytes(n_data, max_batch);
    if (need == 0) return QSG_ERR_ARG;
    if (!d_workspace || workspace_bytes < need || ((uintptr_t)d_workspace % kAlignM) != 0) return QSG_ERR_WORKSPACE;
    qsg_mlp *m = new qsg_mlp();
    carve_mlp((char *)d_workspace, n_data, max_batch, &m->l);
    m->n_data = n_data;
    m->max_batch = max_batch;
    m->st = (cudaStream_t)cuda_stream;
    *out = m;
    return QSG_OK;
}

void qsg_mlp_destroy(qsg_mlp *m) { delete m; }

qsg_status qsg_mlp_set_params(qsg_mlp *m, const float *host) {
    if (!m || !host) return QSG_ERR_ARG;
    const size_t np = (size_t)mlp_param_count();
    MLP_CUDA(cudaMemcpyAsync(m->l.P, host, np * 4, cudaMemcpyHostToDevice, m->st));
    MLP_CUDA(cudaMemsetAsync(m->l.M, 0, np * 4, m->st));
    MLP_CUDA(cudaMemsetAsync(m->l.V, 0, np * 4, m->st));
    MLP_CUDA(cudaStreamSynchronize(m->st));
    m->step = 0;
    m->has_params = true;
    return QSG_OK;
}

qsg_status qsg_mlp_get_params(qsg_mlp *m, float *host) {
    if (!m || !host) return QSG_ERR_ARG;
    if (!m->has_params) return QSG_ERR_STATE;
    MLP_CUDA(cudaMemcpyAsync(host, m->l.P, (size_t)mlp_param_count() * 4, cudaMemcpyDeviceToHost, m->st));
    MLP_CUDA(cudaStreamSynchronize(m->st));
    return QSG_OK;
}

qsg_status qsg_mlp_set_data(qsg_mlp *m, const float *X, const float *T, int64_t n) {
    if (!m || !X || !T || n < 1 || n > m->n_data) return QSG_ERR_ARG;
    MLP_CUDA(cudaMemcpyAsync(m->l.X, X, (size_t)n * 64 * 4, cudaMemcpyHostToDevice, m->st));
    MLP_CUDA(cudaMemcpyAsync(m->l.T, T, (size_t)n * 33 * 4, cudaMemcpyHostToDevice, m->st));
    MLP_CUDA(cudaStreamSynchronize(m->st));
    m->n_loaded = n;
    return QSG_OK;
}

static qsg_status upload_idx(qsg_mlp *m, const int32_t *idx, size_t count) {
    for (size_t i = 0; i < count; ++i)
        if (idx[i] < 0 || idx[i] >= m->n_loaded) return QSG_ERR_ARG;
    MLP_CUDA(cudaMemcpyAsync(m->l.idx, idx, count * 4, cudaMemcpyHostToDevice, m->st));
    return QSG_OK;
}

qsg_status qsg_mlp_grad(qsg_mlp *m, const int32_t *idx, int32_t batch, float *loss, float *grad_host) {
    if (!m || !idx || batch < 1 || batch > m->max_batch) return QSG_ERR_ARG;
    if (!m->has_params || m->n_loaded == 0) return QSG_ERR_STATE;
    qsg_status s = upload_idx(m, idx, (size_t)batch);
    if (s != QSG_OK) return s;
    MLP_CUDA(launch_mlp_step(m->l.P, m->l.M, m->l.V, m->l.X, m->l.T, m->l.idx, batch, m->l.partial, m->l.lossp,
                             m->l.grad, 0, 0.0f, 1, m->l.losses, m->st));
    if (grad_host)
        MLP_CUDA(cudaMemcpyAsync(grad_host, m->l.grad, (size_t)mlp_param_count() * 4, cudaMemcpyDeviceToHost, m->st));
    float l = 0.0f;
    MLP_CUDA(cudaMemcpyAsync(&l, m->l.losses, 4, cudaMemcpyDeviceToHost, m->st));
    MLP_CUDA(cudaStreamSynchronize(m->st));
    if (loss) *loss = l;
    return QSG_OK;
}

qsg_status qsg_mlp_train(qsg_mlp *m, const int32_t *idx, int32_t steps, int32_t batch, float lr, float *losses) {
    if (!m || !idx || steps < 0 || batch < 1 || batch > m->max_batch || !(lr > 0.0f)) return QSG_ERR_ARG;
    if (!m->has_params || m->n_loaded == 0) return QSG_ERR_STATE;
    for (int c0 = 0; c0 < steps; c0 += kChunk) {
        const int nc = steps - c0 < kChunk ? steps - c0 : kChunk;
        qsg_status s = upload_idx(m, idx + (size_t)c0 * batch, (size_t)nc * batch);
        if (s != QSG_OK) return s;
        for (int i = 0; i < nc; ++i) {
            ++m->step;
            MLP_CUDA(launch_mlp_step(m->l.P, m->l.M, m->l.V, m->l.X, m->l.T, m->l.idx + (size_t)i * batch, batch,
                                     m->l.partial, m->l.lossp, nullptr, 1, lr, m->step, m->l.losses + i, m->st));
        }
        if (losses) MLP_CUDA(cudaMemcpyAsync(losses + c0, m->l.losses, (size_t)nc * 4, cudaMemcpyDeviceToHost, m->st));
        // the index buffer is reused by the next chunk
        MLP_CUDA(cudaStreamSynchronize(m->st));
    }
    return QSG_OK;
}

qsg_status qsg_mlp_predict(qsg_mlp *m, const float *X, int64_t n, int32_t bf16, float *Y) {
    if (!m || !X || !Y || n < 1 || n > m->n_data || (bf16 != 0 && bf16 != 1)) return QSG_ERR_ARG;
    if (!m->has_params) return QSG_ERR_STATE;
    MLP_CUDA(cudaMemcpyAsync(m->l.Xp, X, (size_t)n * 64 * 4, cudaMemcpyHostToDevice, m->st));
    MLP_CUDA(launch_mlp_infer(m->l.P, m->l.Pb, m->l.Xp, m->l.Yp, n, bf16, m->st));
    MLP_CUDA(cudaMemcpyAsync(Y, m->l.Yp, (size_t)n * 33 * 4, cudaMemcpyDeviceToHost, m->st));
    MLP_CUDA(cudaStreamSynchronize(m->st));
    return QSG_OK;
}

}  // extern "C"
