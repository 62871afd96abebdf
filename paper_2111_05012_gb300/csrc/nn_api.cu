// C ABI of the learned parallel-transport preconditioner: creation, weights,
// single-layer forward / backward (for parity tests), one Adam training step
// on a batch of (residual, error) pairs.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace {

amg_status nfail(amg_status st, const std::string& m) {
    amg_internal_set_error(m.c_str());
    return st;
}
#define NCK(x)                                                                                       \
    do {                                                                                             \
        cudaError_t e_ = (x);                                                                        \
        if (e_ != cudaSuccess) return nfail(AMG_ECUDA, std::string(#x) + " -> " + cudaGetErrorString(e_)); \
    } while (0)
#define NTRY(x)                       \
    do {                              \
        amg_status s_ = (x);          \
        if (s_ != AMG_OK) return s_;  \
    } while (0)

const int kRev[9] = {0, 5, 6, 7, 8, 1, 2, 3, 4};   // T_d^dag = T_{kRev[d]}

// float -> bfloat16 bits, round to nearest even
uint16_t to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);   // inf / nan
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float from_bf16(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

size_t layer_size(const amg_nn* nn, int l) { return (size_t)nn->ch[l + 1] * nn->ch[l] * 9 * 16 * 2; }

// upload bf16 weights and their adjoint: Wadj[b][a][d'] = W[a][b][rev d']^dag
amg_status upload_weights(amg_nn* nn) {
    for (int l = 0; l < nn->nlayers; ++l) {
        const int cin = nn->ch[l], cout = nn->ch[l + 1];
        const std::vector<float>& w = nn->w[l];
        std::vector<uint16_t> f(layer_size(nn, l)), a(layer_size(nn, l));
        for (size_t i = 0; i < f.size(); ++i) f[i] = to_bf16(w[i]);
        for (int oa = 0; oa < cout; ++oa)
            for (int ib = 0; ib < cin; ++ib)
                for (int d = 0; d < 9; ++d)
                    for (int s = 0; s < 4; ++s)
                        for (int t = 0; t < 4; ++t) {
                            // forward entry W[oa][ib][kRev[d]][t][s] -> adjoint entry Wadj[ib][oa][d][s][t], conjugated
                            size_t src = ((((size_t)oa * cin + ib) * 9 + kRev[d]) * 16 + t * 4 + s) * 2;
                            size_t dst = ((((size_t)ib * cout + oa) * 9 + d) * 16 + s * 4 + t) * 2;
                            a[dst] = f[src];
                            a[dst + 1] = to_bf16(-from_bf16(f[src + 1]));
                        }
        NCK(nn->wbf[l].ensure(f.size() * 2));
        NCK(nn->wadj[l].ensure(a.size() * 2));
        NCK(cudaMemcpy(nn->wbf[l].p, f.data(), f.size() * 2, cudaMemcpyHostToDevice));
        NCK(cudaMemcpy(nn->wadj[l].p, a.data(), a.size() * 2, cudaMemcpyHostToDevice));
    }
    return AMG_OK;
}

const GeomH& geom(amg_nn* nn) { return *amg_internal_geom(nn->d); }
size_t fbytes(amg_nn* nn) { return fine_spinor_bytes(1, geom(nn).V); }

amg_status sum_partials(amg_nn* nn, size_t count, double* out, cudaStream_t s) {
    NCK(cudaMemcpyAsync(nn->hpart, nn->part.p, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < count; ++i) out[i] = nn->hpart[i];
    return AMG_OK;
}

// weight gradient of layer l (Wirtinger, [cout][cin][9][4][4][re,im]) from the
// layer input field (cin channels) and the output gradient (cout channels)
amg_status layer_wgrad(amg_nn* nn, int l, const void* in, const void* gout, std::vector<double>& G, cudaStream_t s) {
    const int cin = nn->ch[l], cout = nn->ch[l + 1];
    const int grid = ptconv_grid();
    const size_t per = (size_t)cout * 16;   // complex per CTA per (b, d)
    NCK(launch_ptconv_wgrad(geom(nn), cin, cout, amg_internal_links(nn->d, 1), in, gout, nn->part.as<double2>(), s));
    std::vector<double> h((size_t)cin * 9 * grid * per * 2);
    NTRY(sum_partials(nn, h.size(), h.data(), s));
    G.assign(layer_size(nn, l), 0.0);
    for (int b = 0; b < cin; ++b)
        for (int d = 0; d < 9; ++d)
            for (int blk = 0; blk < grid; ++blk)
                for (int a = 0; a < cout; ++a)
                    for (int k = 0; k < 16; ++k) {
                        const size_t src = ((((size_t)(b * 9 + d) * grid + blk) * per) + a * 16 + k) * 2;
                        const size_t dst = ((((size_t)a * cin + b) * 9 + d) * 16 + k) * 2;
                        G[dst] += h[src];
                        G[dst + 1] += h[src + 1];
                    }
    return AMG_OK;
}

amg_status ensure_buffers(amg_nn* nn) {
    const size_t fb = fbytes(nn);
    int cmax = 1;
    for (int l = 0; l <= nn->nlayers; ++l) cmax = nn->ch[l] > cmax ? nn->ch[l] : cmax;
    for (int l = 0; l <= nn->nlayers; ++l) NCK(nn->act[l].ensure(fb * nn->ch[l]));
    NCK(nn->gbuf[0].ensure(fb * cmax));
    NCK(nn->gbuf[1].ensure(fb * cmax));
    NCK(nn->ework.ensure(fb));
    size_t pmax = 4096;
    for (int l = 0; l < nn->nlayers; ++l) {
        size_t q = (size_t)nn->ch[l] * 9 * ptconv_grid() * nn->ch[l + 1] * 16 * 2;
        pmax = q > pmax ? q : pmax;
    }
    NCK(nn->part.ensure(pmax * sizeof(double)));
    if (!nn->hpart) NCK(cudaMallocHost(&nn->hpart, pmax * sizeof(double)));
    NCK(nn->canon.ensure((size_t)geom(nn).V * 24 * sizeof(float) * cmax));
    return AMG_OK;
}

}  // namespace

amg_status nn_forward_internal(amg_nn* nn, const void* in32, void* out32, cudaStream_t s) {
    const void* cur = in32;
    for (int l = 0; l < nn->nlayers; ++l) {
        void* dst = (l == nn->nlayers - 1) ? out32 : nn->act[l + 1].p;
        NCK(launch_ptconv_forward(geom(nn), nn->ch[l], nn->ch[l + 1], amg_internal_links(nn->d, 1), nn->wbf[l].p,
                                  cur, dst, s));
        cur = dst;
    }
    return AMG_OK;
}

extern "C" {

amg_status amg_nn_create(amg_dirac* d, int nlayers, const int* channels, const float* weights, amg_nn** out) {
    if (!d || !channels || !weights || !out) return nfail(AMG_EINVAL, "amg_nn_create: NULL argument");
    if (nlayers < 1 || nlayers > AMG_NN_MAX_LAYERS) return nfail(AMG_EINVAL, "amg_nn_create: 1..4 layers");
    if (channels[0] != 1 || channels[nlayers] != 1)
        return nfail(AMG_EINVAL, "amg_nn_create: the network maps one field to one field");
    for (int l = 0; l <= nlayers; ++l)
        if (channels[l] < 1 || channels[l] > 4) return nfail(AMG_EINVAL, "amg_nn_create: 1..4 channels per layer");
    amg_nn* nn = new amg_nn();
    nn->d = d;
    nn->nlayers = nlayers;
    for (int l = 0; l <= nlayers; ++l) nn->ch[l] = channels[l];
    const float* p = weights;
    for (int l = 0; l < nlayers; ++l) {
        size_t n = layer_size(nn, l);
        nn->w.emplace_back(p, p + n);
        nn->m.emplace_back(n, 0.0);
        nn->v.emplace_back(n, 0.0);
        p += n;
    }
    amg_status st = upload_weights(nn);
    if (st == AMG_OK) st = ensure_buffers(nn);
    if (st != AMG_OK) {
        delete nn;
        return st;
    }
    *out = nn;
    return AMG_OK;
}

void amg_nn_destroy(amg_nn* nn) { delete nn; }

amg_status amg_nn_get_weights(amg_nn* nn, int effective, float* host_out) {
    if (!nn || !host_out) return nfail(AMG_EINVAL, "amg_nn_get_weights: NULL argument");
    float* p = host_out;
    for (int l = 0; l < nn->nlayers; ++l) {
        for (size_t i = 0; i < nn->w[l].size(); ++i) p[i] = effective ? from_bf16(to_bf16(nn->w[l][i])) : nn->w[l][i];
        p += nn->w[l].size();
    }
    return AMG_OK;
}

amg_status amg_nn_layer_forward(amg_nn* nn, int layer, const float* in, float* out, amg_stream stream) {
    if (!nn || !in || !out || layer < 0 || layer >= nn->nlayers) return nfail(AMG_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const GeomH& g = geom(nn);
    const int cin = nn->ch[layer], cout = nn->ch[layer + 1];
    NCK(launch_pack_spinor(1, g, in, nn->gbuf[0].p, cin, s));
    NCK(launch_ptconv_forward(g, cin, cout, amg_internal_links(nn->d, 1), nn->wbf[layer].p, nn->gbuf[0].p,
                              nn->gbuf[1].p, s));
    NCK(launch_unpack_spinor(1, g, nn->gbuf[1].p, out, cout, s));
    return AMG_OK;
}

amg_status amg_nn_layer_backward(amg_nn* nn, int layer, const float* in, const float* grad_out, float* grad_in,
                                 double* grad_w, amg_stream stream) {
    if (!nn || !in || !grad_out || layer < 0 || layer >= nn->nlayers) return nfail(AMG_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const GeomH& g = geom(nn);
    const int cin = nn->ch[layer], cout = nn->ch[layer + 1];
    NCK(launch_pack_spinor(1, g, in, nn->gbuf[0].p, cin, s));
    NCK(launch_pack_spinor(1, g, grad_out, nn->gbuf[1].p, cout, s));
    if (grad_w) {
        std::vector<double> G;
        NTRY(layer_wgrad(nn, layer, nn->gbuf[0].p, nn->gbuf[1].p, G, s));
        std::memcpy(grad_w, G.data(), G.size() * sizeof(double));
    }
    if (grad_in) {
        NCK(launch_ptconv_forward(g, cout, cin, amg_internal_links(nn->d, 1), nn->wadj[layer].p, nn->gbuf[1].p,
                                  nn->gbuf[0].p, s));
        NCK(launch_unpack_spinor(1, g, nn->gbuf[0].p, grad_in, cin, s));
    }
    NCK(cudaStreamSynchronize(s));
    return AMG_OK;
}

amg_status amg_nn_apply(amg_nn* nn, const float* in, float* out, amg_stream stream) {
    if (!nn || !in || !out) return nfail(AMG_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const GeomH& g = geom(nn);
    NCK(launch_pack_spinor(1, g, in, nn->act[0].p, 1, s));
    NTRY(nn_forward_internal(nn, nn->act[0].p, nn->ework.p, s));
    NCK(launch_unpack_spinor(1, g, nn->ework.p, out, 1, s));
    return AMG_OK;
}

amg_status amg_nn_train_step(amg_nn* nn, const float* r, const float* e, int npairs, double lr, double* loss_out,
                             amg_stream stream) {
    if (!nn || !r || !e || npairs < 1 || !(lr > 0)) return nfail(AMG_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const GeomH& g = geom(nn);
    const size_t n = (size_t)g.V * 12;   // complex numbers per field
    const int L = nn->nlayers;
    std::vector<std::vector<double>> gsum(L);
    for (int l = 0; l < L; ++l) gsum[l].assign(layer_size(nn, l), 0.0);
    double loss = 0;
    for (int p = 0; p < npairs; ++p) {
        NCK(launch_pack_spinor(1, g, r + (size_t)p * g.V * 24, nn->act[0].p, 1, s));
        for (int l = 0; l < L; ++l)
            NCK(launch_ptconv_forward(g, nn->ch[l], nn->ch[l + 1], amg_internal_links(nn->d, 1), nn->wbf[l].p,
                                      nn->act[l].p, nn->act[l + 1].p, s));
        NCK(launch_pack_spinor(1, g, e + (size_t)p * g.V * 24, nn->ework.p, 1, s));
        // ||e||^2 as the residual of a zero field against e
        double ne2 = 0;
        {
            NCK(cudaMemsetAsync(nn->gbuf[0].p, 0, fbytes(nn), s));
            NCK(launch_residual_scale(nn->gbuf[0].p, nn->ework.p, n, 1.0f, nn->part.as<double>(), s));
            std::vector<double> h(ptconv_grid());
            NTRY(sum_partials(nn, h.size(), h.data(), s));
            for (double x : h) ne2 += x;
        }
        if (!(ne2 > 0)) return nfail(AMG_EINVAL, "amg_nn_train_step: zero error vector");
        // g = (y - e) / ||e||^2 in place of y, and ||y - e||^2
        NCK(launch_residual_scale(nn->act[L].p, nn->ework.p, n, (float)(1.0 / ne2), nn->part.as<double>(), s));
        {
            std::vector<double> h(ptconv_grid());
            NTRY(sum_partials(nn, h.size(), h.data(), s));
            double t = 0;
            for (double x : h) t += x;
            loss += t / ne2;
        }
        if (!std::isfinite(loss)) return nfail(AMG_NAN, "amg_nn_train_step: non-finite loss");
        const void* gout = nn->act[L].p;
        int gi = 0;
        for (int l = L - 1; l >= 0; --l) {
            std::vector<double> G;
            NTRY(layer_wgrad(nn, l, nn->act[l].p, gout, G, s));
            for (size_t i = 0; i < G.size(); ++i) gsum[l][i] += G[i];
            if (l > 0) {
                NCK(launch_ptconv_forward(g, nn->ch[l + 1], nn->ch[l], amg_internal_links(nn->d, 1), nn->wadj[l].p,
                                          gout, nn->gbuf[gi].p, s));
                gout = nn->gbuf[gi].p;
                gi ^= 1;
            }
        }
    }
    // Adam on the real and imaginary parts; d/d(Re W) = 2 Re G, d/d(Im W) = 2 Im G (mean over pairs)
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    nn->adam_t++;
    const double c1 = 1.0 - std::pow(b1, nn->adam_t), c2 = 1.0 - std::pow(b2, nn->adam_t);
    for (int l = 0; l < L; ++l)
        for (size_t i = 0; i < nn->w[l].size(); ++i) {
            const double gr = 2.0 * gsum[l][i] / npairs;
            nn->m[l][i] = b1 * nn->m[l][i] + (1 - b1) * gr;
            nn->v[l][i] = b2 * nn->v[l][i] + (1 - b2) * gr * gr;
            const double mh = nn->m[l][i] / c1, vh = nn->v[l][i] / c2;
            nn->w[l][i] = (float)(nn->w[l][i] - lr * mh / (std::sqrt(vh) + eps));
        }
    NTRY(upload_weights(nn));
    if (loss_out) *loss_out = loss / npairs;
    return AMG_OK;
}

void amg_train_params_default(amg_train_params* p) {
    if (!p) return;
    p->npairs = 4096;
    p->batch = 16;
    p->lr = 1e-3;
    p->seed = 5;
}

amg_status amg_learned_train(amg_hierarchy* h, amg_nn* nn, const amg_train_params* p, double* losses,
                             amg_stream stream) {
    if (!h || !nn || !p || p->npairs < 1 || p->batch < 1 || !(p->lr > 0))
        return nfail(AMG_EINVAL, "amg_learned_train: bad argument");
    amg_dirac* d = amg_internal_hierarchy_dirac(h);
    if (d != nn->d) return nfail(AMG_EINVAL, "amg_learned_train: network and hierarchy use different operators");
    cudaStream_t s = (cudaStream_t)stream;
    const GeomH& g = geom(nn);
    const size_t n = (size_t)g.V * 12;   // complex numbers per field
    const size_t f64 = n * 16, f32 = n * 8;
    DevBuf e0, w, e1, r1, rb, eb;
    NCK(e0.ensure(f64));
    NCK(w.ensure(f64));
    NCK(e1.ensure(f64));
    NCK(r1.ensure(f64));
    NCK(rb.ensure(f32 * p->batch));
    NCK(eb.ensure(f32 * p->batch));
    const int steps = p->npairs / p->batch;
    if (steps < 1) return nfail(AMG_EINVAL, "amg_learned_train: npairs < batch");
    for (int st = 0; st < steps; ++st) {
        for (int q = 0; q < p->batch; ++q) {
            const uint64_t k = (uint64_t)st * p->batch + q;
            // e0: Gaussian field k of stream (seed, AMG_RNG_STREAM_NN); e = e0 - M D e0, r = D e
            NCK(launch_random_normal(p->seed, AMG_RNG_STREAM_NN, k * n, n, e0.as<double>(), s));
            NTRY(amg_apply_D(d, e0.p, w.p, 1, AMG_F64, stream));
            NTRY(amg_precondition(h, w.as<double>(), e1.as<double>(), stream));
            NCK(launch_axpby(0, make_double2(1, 0), e0.p, make_double2(-1, 0), e1.p, n, s));
            NTRY(amg_apply_D(d, e1.p, r1.p, 1, AMG_F64, stream));
            NCK(launch_convert_flat(0, 1, e1.p, (char*)eb.p + q * f32, n, s));
            NCK(launch_convert_flat(0, 1, r1.p, (char*)rb.p + q * f32, n, s));
        }
        double loss = 0;
        NTRY(amg_nn_train_step(nn, rb.as<float>(), eb.as<float>(), p->batch, p->lr, &loss, stream));
        if (losses) losses[st] = loss;
    }
    NCK(cudaStreamSynchronize(s));
    return AMG_OK;
}

}  // extern "C"
