// Checkpoint / resume of a solve: the state image (host only, no device work).
//
// Between iterations IHT carries only the support S, beta on S and its counters
// (Sec. 2.2: the residual, the gradient and the step size are recomputed from
// them every iteration), so this image is all a stopped solve needs to resume
// exactly.  Layout, little-endian, no padding between fields:
//   char     magic[8]   "IHTSTATE"
//   uint32   version    1
//   uint32   header     bytes before the arrays (kStateHeader)
//   int64    n, p       dataset shape the solve ran on
//   int64    n_rows     rows the solve used
//   int32    k, iterations, backtracks, status
//   double   objective, mu
//   uint64   checksum   FNV-1a 64 over the whole image with this field zero
//   int32    support[k] strictly ascending, in [0, p)
//   double   beta_s[k]  finite
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace iht {

constexpr char kStateMagic[8] = {'I', 'H', 'T', 'S', 'T', 'A', 'T', 'E'};
constexpr uint32_t kStateVersion = 1;
constexpr size_t kStateHeader = 8 + 4 + 4 + 3 * 8 + 4 * 4 + 2 * 8 + 8;   // 80 bytes
constexpr size_t kStateChecksumAt = kStateHeader - 8;

static uint64_t fnv1a(const unsigned char *b, size_t n, uint64_t h = 1469598103934665603ull)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

static uint64_t image_checksum(const unsigned char *img, size_t bytes)
{
    static const unsigned char zero[8] = {};
    uint64_t h = fnv1a(img, kStateChecksumAt);
    h = fnv1a(zero, 8, h);
    return fnv1a(img + kStateHeader, bytes - kStateHeader, h);
}

template <typename T>
static void put(unsigned char *&q, T v)
{
    memcpy(q, &v, sizeof(T));
    q += sizeof(T);
}

template <typename T>
static T get(const unsigned char *&q)
{
    T v;
    memcpy(&v, q, sizeof(T));
    q += sizeof(T);
    return v;
}

static bool valid_support(const int32_t *S, const double *b, int32_t k, int64_t p)
{
    for (int32_t c = 0; c < k; ++c) {
        if (S[c] < 0 || S[c] >= p || (c > 0 && S[c] <= S[c - 1])) return false;
        if (!std::isfinite(b[c])) return false;
    }
    return true;
}

}  // namespace iht

using namespace iht;

extern "C" {

int iht_state_bytes(int32_t k, size_t *bytes)
{
    if (!bytes || k < 1 || k > kMaxK) return IHT_EINVAL;
    *bytes = kStateHeader + (size_t)k * (sizeof(int32_t) + sizeof(double));
    return IHT_OK;
}

int iht_state_save(int64_t n, int64_t p, int64_t n_rows, int32_t k, const int32_t *support,
                   const double *beta_s, const iht_result *info, void *buf, size_t buf_bytes)
{
    size_t need = 0;
    if (iht_state_bytes(k, &need) != IHT_OK || !support || !beta_s || !info || !buf) return IHT_EINVAL;
    if (buf_bytes < need || n < 2 || p < 1 || k > p || n_rows < 2 || n_rows > n) return IHT_EINVAL;
    if (!valid_support(support, beta_s, k, p)) return IHT_EINVAL;
    unsigned char *img = static_cast<unsigned char *>(buf);
    unsigned char *q = img;
    memcpy(q, kStateMagic, 8);
    q += 8;
    put<uint32_t>(q, kStateVersion);
    put<uint32_t>(q, (uint32_t)kStateHeader);
    put<int64_t>(q, n);
    put<int64_t>(q, p);
    put<int64_t>(q, n_rows);
    put<int32_t>(q, k);
    put<int32_t>(q, info->iterations);
    put<int32_t>(q, info->backtracks);
    put<int32_t>(q, info->status);
    put<double>(q, info->objective);
    put<double>(q, info->mu);
    put<uint64_t>(q, 0);
    memcpy(q, support, sizeof(int32_t) * (size_t)k);
    q += sizeof(int32_t) * (size_t)k;
    memcpy(q, beta_s, sizeof(double) * (size_t)k);
    const uint64_t h = image_checksum(img, need);
    memcpy(img + kStateChecksumAt, &h, 8);
    return IHT_OK;
}

int iht_state_load(const void *buf, size_t buf_bytes, int32_t k_cap, int64_t *n, int64_t *p,
                   int64_t *n_rows, int32_t *k, int32_t *support, double *beta_s, iht_result *info)
{
    if (!buf || !n || !p || !n_rows || !k || buf_bytes < kStateHeader) return IHT_EINVAL;
    const unsigned char *img = static_cast<const unsigned char *>(buf);
    const unsigned char *q = img;
    if (memcmp(q, kStateMagic, 8) != 0) return IHT_EINVAL;
    q += 8;
    if (get<uint32_t>(q) != kStateVersion || get<uint32_t>(q) != (uint32_t)kStateHeader) return IHT_EINVAL;
    const int64_t nn = get<int64_t>(q), pp = get<int64_t>(q), rr = get<int64_t>(q);
    const int32_t kk = get<int32_t>(q);
    size_t need = 0;
    if (iht_state_bytes(kk, &need) != IHT_OK || buf_bytes != need) return IHT_EINVAL;
    uint64_t stored;
    memcpy(&stored, img + kStateChecksumAt, 8);
    if (stored != image_checksum(img, need)) return IHT_EINVAL;
    if (nn < 2 || pp < 1 || kk > pp || rr < 2 || rr > nn) return IHT_EINVAL;
    const unsigned char *sb = img + kStateHeader;                        // arrays, possibly unaligned:
    const unsigned char *bb = sb + sizeof(int32_t) * (size_t)kk;        // copied out byte-wise
    *n = nn;
    *p = pp;
    *n_rows = rr;
    *k = kk;
    if (!support && !beta_s && !info) return IHT_OK;                 // shape query
    if (!support || !beta_s || kk > k_cap) return IHT_EINVAL;
    memcpy(support, sb, sizeof(int32_t) * (size_t)kk);
    memcpy(beta_s, bb, sizeof(double) * (size_t)kk);
    if (!valid_support(support, beta_s, kk, pp)) return IHT_EINVAL;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iterations = get<int32_t>(q);
        info->backtracks = get<int32_t>(q);
        info->status = get<int32_t>(q);
        info->objective = get<double>(q);
        info->mu = get<double>(q);
    }
    return IHT_OK;
}

}  // extern "C"
