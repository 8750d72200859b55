// Solver checkpoints on storage: a one-line JSON header followed by the raw
// float32 iterate x and momentum point z (include/nufft_radon.h,
// tc_checkpoint_save / tc_checkpoint_load).  Host code only: the arrays go
// through a bounded host staging buffer in chunks, so a checkpoint of a
// 17 GB volume needs no host copy of the whole volume.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

const char kFormat[] = "tc-mbir-checkpoint";
constexpr size_t kStageBytes = (size_t)64 << 20;  // host staging buffer per copy
constexpr size_t kMaxHeader = 4096;

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

// Value of "key": in a one-line JSON object written by save(): the number
// after the colon (strtod accepts the %.17g output), or the first one of an
// array.  false if the key is missing or the value is not a number.
bool json_number(const std::string &h, const char *key, double *out, int index = 0) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = h.find(k);
    if (at == std::string::npos) return false;
    const char *p = h.c_str() + at + k.size();
    while (*p == ' ') ++p;
    if (*p == '[') {
        ++p;
        for (int i = 0; i < index; ++i) {
            p = std::strchr(p, ',');
            if (!p) return false;
            ++p;
        }
    }
    char *end = nullptr;
    const double v = std::strtod(p, &end);
    if (end == p) return false;
    *out = v;
    return true;
}

bool json_int(const std::string &h, const char *key, long long *out) {
    double v;
    if (!json_number(h, key, &v) || v != std::floor(v) || std::fabs(v) > 9.0e15) return false;
    *out = (long long)v;
    return true;
}

// count floats of dev <-> file through the staging buffer
int stream_array(FILE *f, float *dev, size_t count, bool to_file, std::vector<char> &stage, cudaStream_t s) {
    const size_t per = stage.size() / sizeof(float);
    float *h = reinterpret_cast<float *>(stage.data());
    for (size_t off = 0; off < count; off += per) {
        const size_t n = count - off < per ? count - off : per;
        if (to_file) {
            TC_CUDA(cudaMemcpyAsync(h, dev + off, n * sizeof(float), cudaMemcpyDeviceToHost, s));
            TC_CUDA(cudaStreamSynchronize(s));
            if (std::fwrite(h, sizeof(float), n, f) != n) return TC_ERR_INVALID_ARG;
        } else {
            if (std::fread(h, sizeof(float), n, f) != n) return TC_ERR_INVALID_ARG;
            TC_CUDA(cudaMemcpyAsync(dev + off, h, n * sizeof(float), cudaMemcpyHostToDevice, s));
            TC_CUDA(cudaStreamSynchronize(s));
        }
    }
    return TC_OK;
}

bool little_endian() {
    const unsigned one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}

}  // namespace

extern "C" int tc_checkpoint_save(const char *path, const tc_plan *p, const float *x, int batch,
                                  const tc_solve_state *st, void *stream) {
    if (!path || !p || !x || !st || !st->z || batch < 1) return TC_ERR_INVALID_ARG;
    char head[kMaxHeader];
    const int len = std::snprintf(
        head, sizeof(head),
        "{\"format\": \"%s\", \"version\": 1, \"n\": %d, \"n_angles\": %d, \"n_det\": %d, \"batch\": %d, "
        "\"k\": %d, \"n_restarts\": %d, \"t\": %.17g, \"step\": %.17g, \"obj\": [%.17g, %.17g], "
        "\"arrays\": [\"x\", \"z\"], \"dtype\": \"float32\", \"byte_order\": \"%s\"}\n",
        kFormat, p->k.N, p->k.A, p->k.D, batch, st->k, st->n_restarts, st->t, st->step, st->obj[0], st->obj[1],
        little_endian() ? "little" : "big");
    if (len <= 0 || (size_t)len >= sizeof(head)) return TC_ERR_INVALID_ARG;
    File f;
    f.f = std::fopen(path, "wb");
    if (!f.f) return TC_ERR_INVALID_ARG;
    if (std::fwrite(head, 1, (size_t)len, f.f) != (size_t)len) return TC_ERR_INVALID_ARG;
    const size_t count = (size_t)batch * p->k.N * p->k.N;
    std::vector<char> stage(kStageBytes);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = stream_array(f.f, const_cast<float *>(x), count, true, stage, s);
    if (!rc) rc = stream_array(f.f, st->z, count, true, stage, s);
    if (rc) return rc;
    if (std::fflush(f.f) != 0) return TC_ERR_INVALID_ARG;
    return TC_OK;
}

extern "C" int tc_checkpoint_load(const char *path, const tc_plan *p, float *x, int batch,
                                  tc_solve_state *st, void *stream) {
    if (!path || !p || !x || !st || !st->z || batch < 1) return TC_ERR_INVALID_ARG;
    File f;
    f.f = std::fopen(path, "rb");
    if (!f.f) return TC_ERR_INVALID_ARG;
    // header: up to the first newline
    std::string h;
    for (int c; (c = std::fgetc(f.f)) != EOF && c != '\n';) {
        h.push_back((char)c);
        if (h.size() >= kMaxHeader) return TC_ERR_INVALID_ARG;
    }
    if (h.find(std::string("\"format\": \"") + kFormat + "\"") == std::string::npos) return TC_ERR_INVALID_ARG;
    if (h.find(little_endian() ? "\"byte_order\": \"little\"" : "\"byte_order\": \"big\"") == std::string::npos)
        return TC_ERR_INVALID_ARG;
    long long ver, n, a, d, b, k, nr;
    double t, step, o0, o1;
    if (!json_int(h, "version", &ver) || ver != 1 || !json_int(h, "n", &n) || !json_int(h, "n_angles", &a) ||
        !json_int(h, "n_det", &d) || !json_int(h, "batch", &b) || !json_int(h, "k", &k) ||
        !json_int(h, "n_restarts", &nr) || !json_number(h, "t", &t) || !json_number(h, "step", &step) ||
        !json_number(h, "obj", &o0, 0) || !json_number(h, "obj", &o1, 1))
        return TC_ERR_INVALID_ARG;
    if (n != p->k.N || a != p->k.A || d != p->k.D || b != batch || k < 0 || k > 2147483647LL || nr < 0 ||
        nr > 2147483647LL)
        return TC_ERR_INVALID_ARG;
    // the file must hold exactly the two arrays after the header
    const long data_at = std::ftell(f.f);
    const size_t count = (size_t)batch * p->k.N * p->k.N;
    if (data_at < 0 || std::fseek(f.f, 0, SEEK_END) != 0) return TC_ERR_INVALID_ARG;
    const long end = std::ftell(f.f);
    if (end < 0 || (unsigned long long)(end - data_at) != 2ull * count * sizeof(float) ||
        std::fseek(f.f, data_at, SEEK_SET) != 0)
        return TC_ERR_INVALID_ARG;
    std::vector<char> stage(kStageBytes);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = stream_array(f.f, x, count, false, stage, s);
    if (!rc) rc = stream_array(f.f, st->z, count, false, stage, s);
    if (rc) return rc;
    st->k = (int)k;
    st->n_restarts = (int)nr;
    st->t = t;
    st->step = step;
    st->obj[0] = o0;
    st->obj[1] = o1;
    return TC_OK;
}
