// ctf_mlp_host.cu -- C ABI of the learned texel decode: texture creation
// (quantisation to FP16 or FP8 E4M3, then the upload of the stored values:
// FP16 latent grids and the tensor-core operand image), export of the stored
// parameters, and decode of a texel list.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "../../include/ctf.h"
#include "ctf_internal.h"

namespace ctf {
namespace {

int copy_in(const float *src, size_t n, std::vector<float> &dst, const char *what) {
    if (!src) return report(CTF_ERR_ARG, "%s must not be NULL", what);
    dst.resize(n);
    cudaError_t e = cudaMemcpy(dst.data(), src, n * sizeof(float), cudaMemcpyDefault);
    if (e != cudaSuccess) return report_cuda(e, what);
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(dst[i])) return report(CTF_ERR_ARG, "%s[%zu] is not finite", what, i);
    return CTF_OK;
}

uint8_t e4m3(float v) { return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3); }

float e4m3_value(uint8_t b) {
    __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}

}  // namespace

int upload_mlp_texture(ctf_texture_s *t) {
    const bool fp8 = t->mode == CTF_EVAL_MLP_FP8;
    // latents: the stored values are FP16 numbers, so the conversion is exact
    for (int g = 0; g < 2; ++g) {
        const size_t n = t->s_lat[g].size();
        std::vector<__half> h(n);
        for (size_t i = 0; i < n; ++i) h[i] = __float2half_rn(t->s_lat[g][i]);
        cudaError_t e = ctf::dev_malloc(&t->lat[g], n * sizeof(__half));
        if (e == cudaSuccess) e = cudaMemcpy(t->lat[g], h.data(), n * sizeof(__half), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return report_cuda(e, "latent upload");
    }
    // operand image: weights (FP16 or E4M3 numbers, converted exactly), biases, scales
    std::vector<unsigned char> img(kImgBytes, 0);
    auto put_f32 = [&](int off, int i, float v) { std::memcpy(img.data() + off + 4 * i, &v, 4); };
    // FP8: the hidden layers' output scales and biases are multiplied by the
    // inverse activation scale of the next layer's input, so that one FMA
    // gives the next E4M3 operand's value (the scales are positive, so the
    // ReLU commutes with them)
    for (int i = 0; i < kMlpHidden; ++i) {
        put_f32(kImgB1, i, fp8 ? t->s_b1[i] * (1.0f / t->s_ascale[1][i]) : t->s_b1[i]);
        put_f32(kImgB2, i, fp8 ? t->s_b2[i] * (1.0f / t->s_ascale[2][i]) : t->s_b2[i]);
    }
    for (int i = 0; i < kMlpOut; ++i) put_f32(kImgB3, i, t->s_b3[i]);
    const std::vector<float> *S[3] = {&t->s_w1, &t->s_w2, &t->s_w3};
    const int nin[3] = {kMlpIn, kMlpHidden, kMlpHidden};
    const int rows[3] = {kMlpHidden, kMlpHidden, kMlpOut};
    const int imgoff[3] = {kImgW1, kImgW2, kImgW3};
    if (!fp8) {
        const int Kimg[3] = {16, 64, 64};
        for (int l = 0; l < 3; ++l)
            for (int o = 0; o < rows[l]; ++o)
                for (int k = 0; k < nin[l]; ++k) {
                    const __half h = __float2half_rn((*S[l])[(size_t)o * nin[l] + k]);
                    std::memcpy(img.data() + imgoff[l] + core_offset(o, k, Kimg[l], 2), &h, 2);
                }
    } else {
        const int Kimg[3] = {32, 64, 64};
        const int soff[3] = {kImgS1, kImgS2, kImgS3};
        const int aoff[3] = {kImgA1, kImgA2, kImgA3};
        for (int l = 0; l < 3; ++l) {
            for (int k = 0; k < nin[l]; ++k) put_f32(aoff[l], k, 1.0f / t->s_ascale[l][k]);
            for (int o = 0; o < rows[l]; ++o) {
                put_f32(soff[l], o, l < 2 ? t->s_wscale[l][o] * (1.0f / t->s_ascale[l + 1][o]) : t->s_wscale[l][o]);
                for (int k = 0; k < nin[l]; ++k)
                    img[imgoff[l] + core_offset(o, k, Kimg[l], 1)] = e4m3((*S[l])[(size_t)o * nin[l] + k]);
            }
        }
    }
    cudaError_t e = ctf::dev_malloc(&t->img, kImgBytes);
    if (e == cudaSuccess) e = cudaMemcpy(t->img, img.data(), kImgBytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return report_cuda(e, "operand image upload");
    return CTF_OK;
}

MlpDevice mlp_device_view(const ctf_texture_s *t) {
    MlpDevice m;
    for (int g = 0; g < 2; ++g) {
        m.lat[g] = t->lat[g];
        m.gw[g] = t->gw[g];
        m.gh[g] = t->gh[g];
        m.sx[g] = (float)t->gw[g] / (float)t->width;
        m.sy[g] = (float)t->gh[g] / (float)t->height;
    }
    m.img = static_cast<const uint4 *>(t->img);
    m.fp8 = t->mode == CTF_EVAL_MLP_FP8 ? 1 : 0;
    m.err = nullptr;
    if (device_error_word(&m.err) != CTF_OK) m.err = nullptr;  // the index checks then only clamp
    return m;
}

}  // namespace ctf

extern "C" {

int ctf_texture_create_mlp(const ctf_mlp_desc *d, ctf_texture *out) {
    ctf::NvtxRange nvtx_range("ctf_texture_create_mlp");
    using namespace ctf;
    clear_error();
    if (!d || !out) return report(CTF_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (d->mode != CTF_EVAL_MLP_FP16 && d->mode != CTF_EVAL_MLP_FP8)
        return report(CTF_ERR_ARG, "mode %d is not a learned-decode mode", (int)d->mode);
    if (d->width < 1 || d->height < 1 || d->width > 65536 || d->height > 65536)
        return report(CTF_ERR_ARG, "texture %dx%d outside [1, 65536]^2", d->width, d->height);
    for (int g = 0; g < 2; ++g)
        if (d->latent_w[g] < 1 || d->latent_h[g] < 1 || d->latent_w[g] > 16384 || d->latent_h[g] > 16384)
            return report(CTF_ERR_ARG, "latent grid %d is %dx%d, outside [1, 16384]^2", g, d->latent_w[g], d->latent_h[g]);
    const bool fp8 = d->mode == CTF_EVAL_MLP_FP8;
    ctf_texture t = new (std::nothrow) ctf_texture_s();
    if (!t) return report(CTF_ERR_OOM, "host allocation");
    auto bail = [&](int rc) {
        for (int g = 0; g < 2; ++g)
            if (t->lat[g]) ctf::dev_free(t->lat[g]);
        if (t->img) ctf::dev_free(t->img);
        delete t;
        return rc;
    };
    t->width = d->width;
    t->height = d->height;
    t->mode = d->mode;
    cudaGetDevice(&t->device);
    std::vector<float> w1, b1, w2, b2, w3, b3, lat[2], amax[3];
    int rc = CTF_OK;
    const char *names[2] = {"latent[0]", "latent[1]"};
    for (int g = 0; g < 2 && !rc; ++g) {
        t->gw[g] = d->latent_w[g];
        t->gh[g] = d->latent_h[g];
        rc = copy_in(d->latent[g], (size_t)t->gw[g] * t->gh[g] * kMlpCh, lat[g], names[g]);
    }
    if (!rc) rc = copy_in(d->w1, kMlpHidden * kMlpIn, w1, "w1");
    if (!rc) rc = copy_in(d->b1, kMlpHidden, b1, "b1");
    if (!rc) rc = copy_in(d->w2, kMlpHidden * kMlpHidden, w2, "w2");
    if (!rc) rc = copy_in(d->b2, kMlpHidden, b2, "b2");
    if (!rc) rc = copy_in(d->w3, kMlpOut * kMlpHidden, w3, "w3");
    if (!rc) rc = copy_in(d->b3, kMlpOut, b3, "b3");
    const int nin[3] = {kMlpIn, kMlpHidden, kMlpHidden};
    if (!rc && fp8) {
        const char *an[3] = {"act_absmax[0]", "act_absmax[1]", "act_absmax[2]"};
        for (int l = 0; l < 3 && !rc; ++l) rc = copy_in(d->act_absmax[l], nin[l], amax[l], an[l]);
    }
    if (rc) return bail(rc);

    // latents: FP16, round to nearest
    for (int g = 0; g < 2; ++g) {
        t->s_lat[g].resize(lat[g].size());
        for (size_t i = 0; i < lat[g].size(); ++i) t->s_lat[g][i] = __half2float(__float2half_rn(lat[g][i]));
    }
    t->s_b1 = b1;
    t->s_b2 = b2;
    t->s_b3 = b3;
    const std::vector<float> *W[3] = {&w1, &w2, &w3};
    std::vector<float> *S[3] = {&t->s_w1, &t->s_w2, &t->s_w3};
    const int rows[3] = {kMlpHidden, kMlpHidden, kMlpOut};
    if (!fp8) {
        for (int l = 0; l < 3; ++l) {
            S[l]->resize((size_t)rows[l] * nin[l]);
            for (size_t i = 0; i < S[l]->size(); ++i) (*S[l])[i] = __half2float(__float2half_rn((*W[l])[i]));
        }
    } else {
        // activation scales a[k] = absmax / 448 per input channel; weights
        // W'[o][k] = W[o][k] * a[k] scaled per output channel by s[o] =
        // max_k |W'[o][k]| / 448; stored q = e4m3(W' / s).  Then
        // sum_k e4m3(x_k / a_k) * q[o][k] * s[o] approximates (W x)[o].
        for (int l = 0; l < 3; ++l) {
            std::vector<float> a(nin[l]);
            for (int k = 0; k < nin[l]; ++k) {
                const float m = amax[l][k];
                a[k] = m > 0.f ? m / 448.0f : 1.0f;
            }
            t->s_ascale[l] = a;
            S[l]->resize((size_t)rows[l] * nin[l]);
            t->s_wscale[l].resize(rows[l]);
            for (int o = 0; o < rows[l]; ++o) {
                float mx = 0.f;
                for (int k = 0; k < nin[l]; ++k) mx = std::fmax(mx, std::fabs((*W[l])[(size_t)o * nin[l] + k] * a[k]));
                const float s = mx > 0.f ? mx / 448.0f : 1.0f;
                t->s_wscale[l][o] = s;
                for (int k = 0; k < nin[l]; ++k)
                    (*S[l])[(size_t)o * nin[l] + k] = e4m3_value(e4m3((*W[l])[(size_t)o * nin[l] + k] * a[k] / s));
            }
        }
    }
    rc = upload_mlp_texture(t);
    if (rc) return bail(rc);
    *out = t;
    return CTF_OK;
}

int ctf_mlp_export(ctf_texture t, const ctf_mlp_params *p) {
    using namespace ctf;
    clear_error();
    if (!t || !p) return report(CTF_ERR_ARG, "texture and params must not be NULL");
    if (t->mode == CTF_EVAL_BLOCK) return report(CTF_ERR_ARG, "not a learned-decode texture");
    auto put = [](float *dst, const std::vector<float> &src) {
        if (dst && !src.empty()) std::memcpy(dst, src.data(), src.size() * sizeof(float));
    };
    for (int g = 0; g < 2; ++g) put(p->latent[g], t->s_lat[g]);
    put(p->w1, t->s_w1);
    put(p->b1, t->s_b1);
    put(p->w2, t->s_w2);
    put(p->b2, t->s_b2);
    put(p->w3, t->s_w3);
    put(p->b3, t->s_b3);
    for (int l = 0; l < 3; ++l) {
        put(p->weight_scale[l], t->s_wscale[l]);
        put(p->act_scale[l], t->s_ascale[l]);
    }
    return CTF_OK;
}

int ctf_mlp_decode(ctf_texture t, const int32_t *xy, int n, float *out_rgba, void *stream) {
    using namespace ctf;
    clear_error();
    if (!t) return report(CTF_ERR_ARG, "texture is NULL");
    if (t->mode == CTF_EVAL_BLOCK) return report(CTF_ERR_ARG, "not a learned-decode texture");
    if (n < 0) return report(CTF_ERR_ARG, "n = %d is negative", n);
    if (n == 0) return CTF_OK;
    if (!xy || !out_rgba) return report(CTF_ERR_ARG, "xy and out_rgba must not be NULL");
    if ((reinterpret_cast<uintptr_t>(xy) & 7) || (reinterpret_cast<uintptr_t>(out_rgba) & 15))
        return report(CTF_ERR_ALIGN, "xy must be 8-byte and out_rgba 16-byte aligned");
    int *err = nullptr;
    int rc = device_error_word(&err);
    if (rc) return rc;
    cudaError_t e = launch_mlp_decode(mlp_device_view(t), t->width, t->height, reinterpret_cast<const int2 *>(xy), n,
                                      reinterpret_cast<float4 *>(out_rgba), err, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return report_cuda(e, "decode launch");
    return CTF_OK;
}

}  // extern "C"
