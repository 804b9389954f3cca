/* Seeded synthetic graph inputs (host side, plain C) and their CUDA twin.
 *
 * The generators stand in for the paper's datasets (LiveJournal, Twitter2010
 * and the Stanford collection, section 7), which are not available: the
 * directed Erdos-Renyi G(n, m) model and the R-MAT model that section 4's
 * generator table lists.  They emit the raw, unsorted COO edge stream that
 * graph construction consumes: duplicates and self-loops are left in.
 *
 * All functions return 0 on success and a negative value on bad arguments.
 * Host functions write into caller-owned host arrays; the *_dev functions
 * write into caller-owned device arrays on the given CUDA stream.
 */
#ifndef GPR_GEN_H
#define GPR_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* R-MAT quadrant probabilities a, b, c (d = 1 - a - b - c) as the cumulative
 * 32-bit thresholds that gen_rmat_edge compares against. */
int gen_rmat_thresholds(double a, double b, double c, uint32_t* ta, uint32_t* tab, uint32_t* tabc);

/* m_raw independent uniform draws (u, v) over [0, n)^2, slot order. */
int gen_uniform_coo(int32_t n, int64_t m_raw, uint64_t seed, int32_t* src, int32_t* dst);

/* Directed G(n, m): uniform draws in slot order until m distinct pairs with
 * u != v have appeared.  The raw stream (all draws, repeats and loops kept)
 * is written to src/dst (capacity `cap`) and its length to *m_raw.
 * Requires m <= n (n - 1) / 2.  Returns -2 if cap is too small. */
int gen_er_gnm(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst, int64_t cap,
               int64_t* m_raw);

/* Fisher-Yates shuffle of the identity on [0, n) (Durstenfeld's loop from
 * i = n - 1 down to 1, swap with j uniform on [0, i]). */
int gen_permutation(int32_t n, uint64_t seed, int32_t* perm);

/* m_raw R-MAT edge slots over 2^scale ids with rejection of endpoints >= n,
 * then, if perm != NULL, both endpoints mapped through perm. */
int gen_rmat_coo(int scale, int32_t n, int64_t m_raw, double a, double b, double c, uint64_t seed,
                 const int32_t* perm, int32_t* src, int32_t* dst);

/* `count` seed nodes uniform over [0, n), with replacement. */
int gen_seed_nodes(int32_t n, int64_t count, uint64_t seed, int32_t* out);

/* `count` doubles uniform on [0, 1): the top 53 bits of outputs
 * 0..count-1 of stream `stream`, times 2^-53.  Used for workload-level
 * draws (graph sizes, arrival gaps), never for edges. */
int gen_unit_draws(uint64_t seed, uint32_t stream, int64_t count, double* out);

/* CUDA twins: identical bits to the host functions above.  `stream` is a
 * cudaStream_t; perm_dev may be NULL. */
int gen_uniform_coo_dev(int32_t n, int64_t m_raw, uint64_t seed, int32_t* src_dev,
                        int32_t* dst_dev, void* stream);
int gen_rmat_coo_dev(int scale, int32_t n, int64_t m_raw, double a, double b, double c,
                     uint64_t seed, const int32_t* perm_dev, int32_t* src_dev, int32_t* dst_dev,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GPR_GEN_H */
