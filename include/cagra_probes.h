/*
 * cagra_probes — measurement probes of the benchmark (not part of the
 * product library libcagra_gb.so): the roofline denominators of the gathers,
 * measured on the GPU at hand.  Built into libcagra_probes.so from
 * paper_1608_01362_gb300/probes/.  Status codes and conventions as in
 * cagra_gb.h.
 */
#ifndef CAGRA_PROBES_H
#define CAGRA_PROBES_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Roofline denominators measured on the current GPU (the gathers of
 * Algorithm 3 and of the CF / batched-PPR forms are bound by random reads,
 * not by a streaming copy).
 *
 * cg_measure_row_gather: a grid of two 1024-thread blocks per SM reads rows
 * of row_bytes (4, 128 or 256) at random positions (a fixed LCG, 4 rows in
 * flight per reading group; 32 bytes per lane for rows of 128 and 256) from
 * a zeroed device table of table_bytes (at least two rows, at most 8 GiB;
 * the rows used are the largest power of two that fits).  Writes the bytes
 * read per second (average of 3 launches after one warm-up) to
 * *bytes_per_s.  A table that fits in L2 measures L2's random-row rate, a
 * larger one HBM's.  Allocates and frees the table (cudaMalloc / cudaFree);
 * synchronizes the stream.  CG_ERR_INVALID_ARG for other sizes.
 *
 * cg_measure_smem_lookups: one 1024-thread block per SM looks up random
 * 4-byte entries of a 128 KB shared-memory table, 16 in flight per thread;
 * writes lookups per second (whole GPU) to *lookups_per_s.  Synchronizes.
 */
int cg_measure_row_gather(int32_t row_bytes, int64_t table_bytes,
                          double *bytes_per_s, cudaStream_t stream);
int cg_measure_smem_lookups(double *lookups_per_s, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CAGRA_PROBES_H */
