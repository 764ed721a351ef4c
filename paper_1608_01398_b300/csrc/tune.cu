// Autotuner for the gradient passes' launch shapes.
//
// The passes have knobs that change only how data is staged, never the
// arithmetic (TMA stages per warpgroup in the single-column pass; genotype
// stages, the buffer-pair mode and the finalisation width in the multi-column
// pass), so every candidate writes the same bits.  The pass modules run the
// candidates on the first pass of a key (device, padded samples, SNPs, pass
// kind, accumulator-width bucket) and store the fastest here; later passes,
// including those captured into graphs, read it back.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "common.cuh"

namespace iht {

namespace {

using Key = std::tuple<int, int64_t, int64_t, int, int>;   // device, n_pad, p, kind, bucket

struct Choice {
    int params[kTuneParams];
    double ms;          // time of the chosen shape (0: pinned)
    int candidates;     // timed runs (0: pinned)
};

std::mutex g_tune_mu;
std::map<Key, Choice> g_tune;
int g_tune_on = -1;     // -1: not read from the environment yet

Key key_of(const iht_dataset *ds, int kind, int bucket)
{
    return Key(ds->ctx->device, ds->n_pad, ds->p, kind, bucket);
}

}  // namespace

bool autotune_enabled()
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_tune_on < 0) {
        const char *e = getenv("IHT_AUTOTUNE");
        g_tune_on = (e && e[0] == '0') ? 0 : 1;
    }
    return g_tune_on == 1;
}

bool tune_lookup(const iht_dataset *ds, int kind, int bucket, int *params)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key_of(ds, kind, bucket));
    if (it == g_tune.end()) return false;
    memcpy(params, it->second.params, sizeof(it->second.params));
    return true;
}

void tune_store(const iht_dataset *ds, int kind, int bucket, const int *params, double ms, int candidates)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    Choice c{};
    memcpy(c.params, params, sizeof(c.params));
    c.ms = ms;
    c.candidates = candidates;
    g_tune[key_of(ds, kind, bucket)] = c;
}

bool stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

// Host-side validation and bucket of a (kind, ncols) pair: the bucket, or -1
// when the kind or the shape does not fit the pass.
static int tune_bucket_checked(const iht_dataset *ds, int kind, int ncols, const int *params)
{
    if (kind == IHT_PASS_SINGLE) {
        if (ncols != 1) return -1;
        return (!params || grad_tc_shape_fits(ds, params)) ? 0 : -1;
    }
    if (kind == IHT_PASS_MULTI) {
        if (ncols < 1) return -1;
        return (!params || grad_mrhs_shape_fits(ncols, params)) ? grad_mrhs_bucket(ncols) : -1;
    }
    return -1;
}

static int tune_nparams(int kind) { return kind == IHT_PASS_SINGLE ? 1 : 5; }

}  // namespace iht

using namespace iht;

extern "C" {

void iht_set_autotune(int on)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_on = on ? 1 : 0;
}

void iht_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

int iht_tune_pin(const iht_dataset *ds, int32_t kind, int32_t ncols, const int32_t *params, int32_t nparams)
{
    if (!ds || !params || (kind != IHT_PASS_SINGLE && kind != IHT_PASS_MULTI) || nparams != tune_nparams(kind))
        return IHT_EINVAL;
    int prm[kTuneParams] = {};
    for (int i = 0; i < nparams; ++i) prm[i] = params[i];
    const int bucket = tune_bucket_checked(ds, kind, ncols, prm);
    if (bucket < 0) return IHT_EINVAL;
    tune_store(ds, kind, bucket, prm, 0.0, 0);
    return IHT_OK;
}

int iht_tune_query(const iht_dataset *ds, int32_t kind, int32_t ncols, int32_t *params, int32_t nparams)
{
    if (!ds || !params || (kind != IHT_PASS_SINGLE && kind != IHT_PASS_MULTI) || nparams != tune_nparams(kind))
        return IHT_EINVAL;
    const int bucket = tune_bucket_checked(ds, kind, ncols, nullptr);
    if (bucket < 0) return IHT_EINVAL;
    int prm[kTuneParams];
    if (!tune_lookup(ds, kind, bucket, prm)) return IHT_EAGAIN;
    for (int i = 0; i < nparams; ++i) params[i] = prm[i];
    return IHT_OK;
}

int iht_tuning_summary(char *buf, size_t buf_bytes)
{
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto &kv : g_tune) {
            const Key &k = kv.first;
            const Choice &c = kv.second;
            char line[256];
            const char *how = c.candidates ? "tuned" : "pinned";
            if (std::get<3>(k) == IHT_PASS_SINGLE)
                snprintf(line, sizeof line,
                         "single-column device %d n_pad %lld p %lld: tma_stages %d (%s, %.3f ms, %d runs)\n",
                         std::get<0>(k), (long long)std::get<1>(k), (long long)std::get<2>(k), c.params[0],
                         how, c.ms, c.candidates);
            else
                snprintf(line, sizeof line,
                         "multi-column device %d n_pad %lld p %lld N<=%d: tiles %d genotype_stages %d "
                         "pairs %d finalise8 %d padded %d (%s, %.3f ms, %d runs)\n",
                         std::get<0>(k), (long long)std::get<1>(k), (long long)std::get<2>(k), std::get<4>(k),
                         c.params[4], c.params[0], c.params[1], c.params[2], c.params[3], how, c.ms,
                         c.candidates);
            out += line;
        }
    }
    if (!buf) return (int)out.size() + 1;
    if (buf_bytes == 0) return IHT_EINVAL;
    const size_t m = std::min(out.size(), buf_bytes - 1);
    memcpy(buf, out.data(), m);
    buf[m] = '\0';
    return IHT_OK;
}

}  // extern "C"
