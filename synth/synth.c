/*
 * Seeded synthetic genotype generator.
 *
 * This file is input generation only: it draws genotype codes from a
 * counter-based hash and writes them in the PLINK .bed SNP-major 2-bit
 * layout.  It holds none of the method's arithmetic (no standardisation,
 * no products, no selection).  The oracle tests, the GPU tests and the
 * benchmark all draw their inputs through it, so both sides of every parity
 * check see byte-identical genotypes.
 *
 * Draw for SNP j, sample i:
 *   s_j = splitmix64(seed + j * 0xD1B54A32D192ED03)
 *   h   = splitmix64(s_j + i)
 *   code = 1 (missing)          if (uint32)h        <  tmiss
 *        = 0 (hom-ref, dosage 0) else if (h >> 32)  <  t0[j]
 *        = 2 (het,     dosage 1) else if (h >> 32)  <  t1[j]
 *        = 3 (hom-alt, dosage 2) otherwise
 * splitmix64 is Steele, Lea & Flood's published 64-bit mixer (OOPSLA 2014).
 * The thresholds t0, t1 (Hardy-Weinberg proportions of a per-SNP allele
 * frequency) and tmiss are computed by the caller.
 *
 * .bed body layout: SNP j occupies row_bytes bytes; sample i sits in bits
 * 2*(i%4) .. 2*(i%4)+1 of byte i/4.  Pad bits of the last byte and pad bytes
 * up to row_bytes are zero (the PLINK convention).
 */
#include <stdint.h>
#include <string.h>

static inline uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline int draw_code(uint64_t sj, int64_t i, uint32_t t0, uint32_t t1, uint32_t tmiss)
{
    uint64_t h = splitmix64(sj + (uint64_t)i);
    uint32_t lo = (uint32_t)h, hi = (uint32_t)(h >> 32);
    if (lo < tmiss) return 1;
    if (hi < t0) return 0;
    if (hi < t1) return 2;
    return 3;
}

static inline uint64_t snp_stream(uint64_t seed, int64_t j)
{
    return splitmix64(seed + (uint64_t)j * 0xD1B54A32D192ED03ull);
}

/* Fill SNP rows [snp_begin, snp_end) of a .bed body (no magic header). */
void synth_bed_body(uint8_t *out, int64_t n, int64_t snp_begin, int64_t snp_end,
                    int64_t row_bytes, uint64_t seed, const uint32_t *t0,
                    const uint32_t *t1, uint32_t tmiss)
{
    const int64_t nb = (n + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t j = snp_begin; j < snp_end; ++j) {
        uint8_t *row = out + (j - snp_begin) * row_bytes;
        const uint64_t sj = snp_stream(seed, j);
        for (int64_t b = 0; b < nb; ++b) {
            unsigned byte = 0;
            for (int q = 0; q < 4; ++q) {
                int64_t i = 4 * b + q;
                if (i < n) byte |= (unsigned)draw_code(sj, i, t0[j], t1[j], tmiss) << (2 * q);
            }
            row[b] = (uint8_t)byte;
        }
        if (row_bytes > nb) memset(row + nb, 0, (size_t)(row_bytes - nb));
    }
}

/* Codes (0..3) of m listed SNPs, out is m x n, row-major by SNP. */
void synth_codes(int8_t *out, int64_t n, const int64_t *snps, int64_t m, uint64_t seed,
                 const uint32_t *t0, const uint32_t *t1, uint32_t tmiss)
{
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < m; ++a) {
        const int64_t j = snps[a];
        const uint64_t sj = snp_stream(seed, j);
        for (int64_t i = 0; i < n; ++i)
            out[a * n + i] = (int8_t)draw_code(sj, i, t0[j], t1[j], tmiss);
    }
}
