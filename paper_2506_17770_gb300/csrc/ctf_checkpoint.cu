// ctf_checkpoint.cu -- texture checkpoints (save and rebuild a block or
// learned texture bit for bit), one-call training of a learned texture, and
// the stream-status entry point.
//
// A learned texture is rebuilt from its stored values (FP16 or E4M3 numbers
// held as floats, FP32 biases and scales), so loading does no quantisation
// and the operand image comes out byte for byte as the saved texture's.
// Loading parses and checks the whole file, down to every stored value being
// a number of its format, before any device work.
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "../../include/ctf.h"
#include "ctf_internal.h"

namespace ctf {
namespace {

constexpr char kTexMagic[8] = {'C', 'T', 'F', 'T', 'E', 'X', '0', '1'};
constexpr uint32_t kTexVersion = 1;
constexpr size_t kTexHead = 8 + 4 + 7 * 4;  // magic, version, mode, width, height, 4 latent sides

// Sizes of the float arrays of a learned texture, in file order.
std::vector<size_t> mlp_sizes(int mode, const int32_t lat[4]) {
    std::vector<size_t> n = {(size_t)lat[0] * lat[1] * kMlpCh, (size_t)lat[2] * lat[3] * kMlpCh,
                             (size_t)kMlpHidden * kMlpIn, kMlpHidden, (size_t)kMlpHidden * kMlpHidden, kMlpHidden,
                             (size_t)kMlpOut * kMlpHidden, kMlpOut};
    if (mode == CTF_EVAL_MLP_FP8) {
        for (size_t s : {(size_t)kMlpHidden, (size_t)kMlpHidden, (size_t)kMlpOut}) n.push_back(s);  // weight scales
        for (size_t s : {(size_t)kMlpIn, (size_t)kMlpHidden, (size_t)kMlpHidden}) n.push_back(s);   // activation scales
    }
    return n;
}

// The stored arrays of a learned texture, in the order of mlp_sizes.
std::vector<std::vector<float> *> mlp_arrays(ctf_texture_s *t) {
    std::vector<std::vector<float> *> a = {&t->s_lat[0], &t->s_lat[1], &t->s_w1, &t->s_b1,
                                           &t->s_w2,     &t->s_b2,     &t->s_w3, &t->s_b3};
    if (t->mode == CTF_EVAL_MLP_FP8) {
        for (int l = 0; l < 3; ++l) a.push_back(&t->s_wscale[l]);
        for (int l = 0; l < 3; ++l) a.push_back(&t->s_ascale[l]);
    }
    return a;
}

// Whether every stored value of a learned texture is what its format
// holds: FP16 numbers (latents, and the weights of an FP16 texture), E4M3
// numbers (the weights of an FP8 texture), finite biases and positive
// finite scales.
bool stored_values_valid(ctf_texture_s *t) {
    auto is_half = [](float v) { return std::isfinite(v) && __half2float(__float2half_rn(v)) == v; };
    auto is_e4m3 = [](float v) {
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        return std::isfinite(v) && __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))) == v;
    };
    const bool fp8 = t->mode == CTF_EVAL_MLP_FP8;
    for (int g = 0; g < 2; ++g)
        for (float v : t->s_lat[g])
            if (!is_half(v)) return false;
    for (const std::vector<float> *w : {&t->s_w1, &t->s_w2, &t->s_w3})
        for (float v : *w)
            if (!(fp8 ? is_e4m3(v) : is_half(v))) return false;
    for (const std::vector<float> *b : {&t->s_b1, &t->s_b2, &t->s_b3})
        for (float v : *b)
            if (!std::isfinite(v)) return false;
    if (fp8)
        for (int l = 0; l < 3; ++l)
            for (const std::vector<float> *sc : {&t->s_wscale[l], &t->s_ascale[l]})
                for (float v : *sc)
                    if (!(std::isfinite(v) && v > 0.f)) return false;
    return true;
}

}  // namespace
}  // namespace ctf

extern "C" {

int ctf_checkpoint_save(ctf_texture t, const char *path) {
    using namespace ctf;
    clear_error();
    if (!t || !path) return report(CTF_ERR_ARG, "texture and path must not be NULL");
    std::vector<unsigned char> payload;
    const bool block = t->mode == CTF_EVAL_BLOCK;
    int32_t lat[4] = {0, 0, 0, 0};
    if (block) {
        payload.resize((size_t)(t->width / 4) * (size_t)(t->height / 4) * 8);
        cudaError_t e = cudaMemcpy(payload.data(), t->blocks, payload.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return report_cuda(e, "reading the blocks");
    } else {
        lat[0] = t->gw[0];
        lat[1] = t->gh[0];
        lat[2] = t->gw[1];
        lat[3] = t->gh[1];
        const std::vector<size_t> n = mlp_sizes(t->mode, lat);
        const std::vector<std::vector<float> *> a = mlp_arrays(t);
        for (size_t i = 0; i < a.size(); ++i) {
            if (a[i]->size() != n[i]) return report(CTF_ERR_ARG, "texture has no stored parameters");
            const unsigned char *b = reinterpret_cast<const unsigned char *>(a[i]->data());
            payload.insert(payload.end(), b, b + n[i] * sizeof(float));
        }
    }
    std::vector<unsigned char> all(kTexHead);
    const int32_t head[7] = {(int32_t)t->mode, t->width, t->height, lat[0], lat[1], lat[2], lat[3]};
    std::memcpy(all.data(), kTexMagic, 8);
    std::memcpy(all.data() + 8, &kTexVersion, 4);
    std::memcpy(all.data() + 12, head, sizeof(head));
    all.insert(all.end(), payload.begin(), payload.end());
    const uint64_t h = fnv1a(all.data(), all.size());
    const unsigned char *hb = reinterpret_cast<const unsigned char *>(&h);
    all.insert(all.end(), hb, hb + 8);
    FILE *f = std::fopen(path, "wb");
    if (!f) return report(CTF_ERR_ARG, "cannot open %s for writing", path);
    bool ok = std::fwrite(all.data(), 1, all.size(), f) == all.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return report(CTF_ERR_ARG, "writing %s failed", path);
    return CTF_OK;
}

int ctf_checkpoint_load(const char *path, ctf_texture *out) {
    using namespace ctf;
    clear_error();
    if (!path || !out) return report(CTF_ERR_ARG, "path and out must not be NULL");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return report(CTF_ERR_ARG, "cannot open %s", path);
    std::vector<unsigned char> all;
    unsigned char tmp[65536];
    size_t k;
    while ((k = std::fread(tmp, 1, sizeof(tmp), f)) > 0) all.insert(all.end(), tmp, tmp + k);
    std::fclose(f);
    const size_t head = kTexHead;
    if (all.size() < head + 8 || std::memcmp(all.data(), kTexMagic, 8) != 0)
        return report(CTF_ERR_CORRUPT, "%s is not a texture checkpoint", path);
    uint64_t stored = 0;
    std::memcpy(&stored, all.data() + all.size() - 8, 8);
    if (fnv1a(all.data(), all.size() - 8) != stored) return report(CTF_ERR_CORRUPT, "checksum mismatch in %s", path);
    uint32_t ver = 0;
    int32_t h[7];
    std::memcpy(&ver, all.data() + 8, 4);
    std::memcpy(h, all.data() + 12, sizeof(h));
    if (ver != kTexVersion) return report(CTF_ERR_CORRUPT, "texture checkpoint version %u, expected %u", ver, kTexVersion);
    const int mode = h[0], W = h[1], H = h[2];
    const unsigned char *payload = all.data() + head;
    const size_t pbytes = all.size() - head - 8;
    if (mode == CTF_EVAL_BLOCK) {
        if (W < 4 || H < 4 || W > 65536 || H > 65536 || W % 4 || H % 4)
            return report(CTF_ERR_CORRUPT, "block texture %dx%d in %s", W, H, path);
        if (pbytes != (size_t)(W / 4) * (size_t)(H / 4) * 8)
            return report(CTF_ERR_CORRUPT, "%s holds %zu bytes of blocks for a %dx%d texture", path, pbytes, W, H);
        ctf_texture_desc d;
        std::memset(&d, 0, sizeof(d));
        d.width = W;
        d.height = H;
        d.mode = CTF_EVAL_BLOCK;
        d.blocks = payload;
        return ctf_texture_create(&d, out);
    }
    if (mode != CTF_EVAL_MLP_FP16 && mode != CTF_EVAL_MLP_FP8)
        return report(CTF_ERR_CORRUPT, "texture mode %d in %s", mode, path);
    if (W < 1 || H < 1 || W > 65536 || H > 65536) return report(CTF_ERR_CORRUPT, "texture %dx%d in %s", W, H, path);
    for (int i = 0; i < 4; ++i)
        if (h[3 + i] < 1 || h[3 + i] > 16384) return report(CTF_ERR_CORRUPT, "latent grid side %d in %s", h[3 + i], path);
    const std::vector<size_t> n = mlp_sizes(mode, h + 3);
    size_t want = 0;
    for (size_t s : n) want += s * sizeof(float);
    if (pbytes != want) return report(CTF_ERR_CORRUPT, "%s holds %zu bytes of parameters, expected %zu", path, pbytes, want);
    ctf_texture t = new (std::nothrow) ctf_texture_s();
    if (!t) return report(CTF_ERR_OOM, "host allocation");
    t->width = W;
    t->height = H;
    t->mode = (ctf_eval_mode)mode;
    t->gw[0] = h[3];
    t->gh[0] = h[4];
    t->gw[1] = h[5];
    t->gh[1] = h[6];
    cudaGetDevice(&t->device);
    const std::vector<std::vector<float> *> a = mlp_arrays(t);
    size_t off = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        a[i]->resize(n[i]);
        std::memcpy(a[i]->data(), payload + off, n[i] * sizeof(float));
        off += n[i] * sizeof(float);
    }
    if (!stored_values_valid(t)) {
        delete t;
        return report(CTF_ERR_CORRUPT, "%s holds values its format cannot store", path);
    }
    const int rc = upload_mlp_texture(t);
    if (rc) {
        for (int g = 0; g < 2; ++g)
            if (t->lat[g]) ctf::dev_free(t->lat[g]);
        if (t->img) ctf::dev_free(t->img);
        delete t;
        return rc;
    }
    *out = t;
    return CTF_OK;
}

int ctf_mlp_train(ctf_texture exact_src, const ctf_train_desc *desc, ctf_eval_mode mode, ctf_texture *out_mlp,
                  ctf_train_report *rep, void *stream) {
    ctf::NvtxRange nvtx_range("ctf_mlp_train");
    using namespace ctf;
    clear_error();
    if (!desc || !out_mlp) return report(CTF_ERR_ARG, "desc and out_mlp must not be NULL");
    *out_mlp = nullptr;
    if (mode != CTF_EVAL_MLP_FP16 && mode != CTF_EVAL_MLP_FP8)
        return report(CTF_ERR_ARG, "mode %d is not a learned-decode mode", (int)mode);
    ctf_trainer tr = nullptr;
    int rc = ctf_trainer_create(exact_src, desc, &tr);
    if (rc) return rc;
    const auto t0 = std::chrono::steady_clock::now();
    rc = ctf_trainer_step(tr, desc->total_steps, stream);
    if (!rc) rc = ctf_sync_check(stream);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    ctf_texture out = nullptr;
    if (!rc) rc = ctf_trainer_export(tr, mode, &out);
    double mse = 0.0, mx = 0.0;
    if (!rc) rc = ctf_texture_compare(exact_src, out, &mse, &mx, stream);
    const std::string msg = rc ? ctf_last_error() : "";
    ctf_trainer_destroy(tr);
    if (rc) {
        if (out) ctf_texture_destroy(out);
        return report(rc, "%s", msg.c_str());
    }
    if (rep) {
        rep->steps = desc->total_steps;
        rep->texels = desc->total_steps * (int64_t)desc->batch;
        rep->seconds = secs;
        rep->mse_rgb = mse;
        rep->max_abs = mx;
        rep->psnr_db = mse > 0.0 ? -10.0 * std::log10(mse) : INFINITY;
    }
    *out_mlp = out;
    return CTF_OK;
}

int ctf_stream_status(void *stream) { return ctf_sync_check(stream); }

}  // extern "C"
