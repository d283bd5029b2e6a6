// tune.cu -- tile-shape autotuner with an on-disk cache.
//
// Each built column-tile variant of the hydro kernel (all give the same
// result bits) is timed on a synthetic mesh of the requested block geometry
// through the persistent batch path; the fastest is returned and cached in a
// JSON file keyed by (GPU name, ndim, block size, task). The paper's
// conclusion names auto-tuned kernel generation as future work for ORCHA;
// this is the runtime form of it for the one kernel here.
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/orcha.h"
#include "launch.h"
#include "runtime.h"

namespace {

using Cache = std::map<std::string, std::vector<double>>;

// The cache file holds one entry per line: "key": [tx, ty, ms_per_step],
Cache read_cache(const char* path) {
    Cache c;
    if (!path) return c;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1), b0 = line.find('[', q1), b1 = line.find(']', b0);
        if (q0 == std::string::npos || q1 == std::string::npos || b0 == std::string::npos || b1 == std::string::npos)
            continue;
        std::vector<double> v;
        std::stringstream ss(line.substr(b0 + 1, b1 - b0 - 1));
        std::string tok;
        while (std::getline(ss, tok, ',')) v.push_back(atof(tok.c_str()));
        if (v.size() >= 2) c[line.substr(q0 + 1, q1 - q0 - 1)] = v;
    }
    return c;
}

bool write_cache(const char* path, const Cache& c) {
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return false;
        f << "{\n";
        size_t i = 0;
        for (auto& kv : c) {
            f << "  \"" << kv.first << "\": [";
            for (size_t j = 0; j < kv.second.size(); ++j) f << (j ? ", " : "") << kv.second[j];
            f << "]" << (++i < c.size() ? "," : "") << "\n";
        }
        f << "}\n";
    }
    return std::rename(tmp.c_str(), path) == 0;
}

}  // namespace

extern "C" orcha_status orcha_autotune(int32_t ndim, const int32_t bs[3], orcha_task task, int32_t nblocks,
                                       const char* cache_path, int32_t* tx_out, int32_t* ty_out, double* ms_out) {
    if (!bs || !tx_out || !ty_out) return orcha::set_error(ORCHA_ERR_INVALID, "autotune: null argument");
    if (!orcha::is_step_task(task))
        return orcha::set_error(ORCHA_ERR_INVALID, "autotune: task must be a whole-step hydro task");
    if (nblocks < 1 || nblocks > (1 << 16)) return orcha::set_error(ORCHA_ERR_INVALID, "autotune: nblocks in [1, 65536]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return orcha::cuda_error(e, "autotune: cudaGetDevice");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return orcha::cuda_error(e, "autotune: device properties");
    char key[512];
    snprintf(key, sizeof(key), "%s|ndim=%d|bs=%dx%dx%d|task=%d", prop.name, ndim, bs[0], bs[1], ndim == 3 ? bs[2] : 1,
             (int)task);
    Cache cache = read_cache(cache_path);
    auto hit = cache.find(key);
    if (hit != cache.end()) {
        *tx_out = (int32_t)hit->second[0];
        *ty_out = (int32_t)hit->second[1];
        if (ms_out) *ms_out = hit->second.size() > 2 ? hit->second[2] : -1.0;
        return ORCHA_OK;
    }

    // synthetic mesh of about nblocks blocks, as cubic as possible
    orcha_mesh_desc d{};
    d.ndim = ndim;
    const int n = ndim == 3 ? (int)std::ceil(std::cbrt((double)nblocks) - 1e-9) : (int)std::ceil(std::sqrt((double)nblocks) - 1e-9);
    for (int a = 0; a < 3; ++a) {
        d.nb[a] = a < ndim ? n : 1;
        d.bs[a] = a < ndim ? bs[a] : 1;
        d.lo[a] = 0.0;
        d.hi[a] = 1.0;
        d.periodic[a] = 1;
    }
    d.gamma = 1.4;
    d.cfl = 0.8;
    const size_t elems = orcha_state_elems(&d);
    if (elems == 0) return orcha::set_error(ORCHA_ERR_INVALID, "autotune: invalid block geometry");
    double* buf = nullptr;
    e = cudaMalloc(&buf, sizeof(double) * (2 * elems + 1));
    if (e != cudaSuccess) return orcha::cuda_error(e, "autotune: buffers");
    d.state_dev[0] = buf;
    d.state_dev[1] = buf + elems;
    d.dt_dev = buf + 2 * elems;
    orcha_mesh* mesh = nullptr;
    orcha_packet* pk = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    orcha_status s = orcha_mesh_create(&d, &mesh);
    std::vector<int32_t> ids;
    int best_tx = 0, best_ty = 0;
    double best_ms = 1e300;
    if (!s) {
        const int nb = d.nb[0] * d.nb[1] * d.nb[2];
        for (int i = 0; i < nb; ++i) ids.push_back(i);
        s = orcha_packet_create(mesh, ids.data(), nb, &pk);
    }
    if (!s) {
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(double) * 2 * elems, st);
        if (e != cudaSuccess) s = orcha::cuda_error(e, "autotune: setup");
    }
    if (!s) {
        for (auto& t : orcha::kTiles) {
            if (bs[0] % t[0] || bs[1] % t[1]) continue;
            // the same input for every candidate
            e = orcha::launch_synthetic_state(mesh->dev, d.state_dev[mesh->cur], st);
            if (e != cudaSuccess) { s = orcha::cuda_error(e, "autotune: state"); break; }
            orcha_batch* b = nullptr;
            if ((s = orcha_batch_create(&pk, 1, t[0], t[1], &b))) break;
            // two-step launches need even step counts
            const bool pairs = orcha::prec_is_tb2(orcha::prec_of(task));
            const int warm = 2, steps = pairs ? 6 : 5;
            s = orcha_batch_advance(b, task, warm, 1, 0, st);
            if (!s) e = cudaEventRecord(e0, st);
            if (!s && e == cudaSuccess) s = orcha_batch_advance(b, task, steps, 0, 0, st);
            if (!s && e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (!s && e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (!s && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            orcha_batch_destroy(b);
            if (s) break;
            if (e != cudaSuccess) { s = orcha::cuda_error(e, "autotune: timing"); break; }
            const double per = ms / steps;
            if (per < best_ms) { best_ms = per; best_tx = t[0]; best_ty = t[1]; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    orcha_packet_destroy(pk);
    orcha_mesh_destroy(mesh);
    cudaFree(buf);
    if (s) return s;
    if (best_tx == 0) return orcha::set_error(ORCHA_ERR_UNSUPPORTED, "autotune: no tile variant divides the block");
    *tx_out = best_tx;
    *ty_out = best_ty;
    if (ms_out) *ms_out = best_ms;
    if (cache_path) {
        cache[key] = {(double)best_tx, (double)best_ty, best_ms};
        if (!write_cache(cache_path, cache)) return orcha::set_error(ORCHA_ERR_INVALID, "autotune: cannot write the cache file");
    }
    return ORCHA_OK;
}
