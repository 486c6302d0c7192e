/*
 * dtbgen.h -- C ABI of the seeded synthetic network generator (the input
 * generator shared by the tests' oracle inputs and the GPU library's inputs).
 *
 * The paper builds its network from subject sMRI/DTI/PET data (section III.B,
 * Table I), which is not available; the generator draws a stand-in with the
 * same structure: heterogeneous voxel sizes, 80/20 E/I, fixed in-degree,
 * multiple edges allowed, no self loops, intra-voxel inputs plus excitatory
 * long-range inputs chosen by a row-normalised DTI-like voxel matrix.  Each
 * synapse is a pure function of (seed, postsynaptic neuron, input slot), so
 * host (libdtbgen_host.so) and device (libdtbgen_dev.so) agree bit for bit.
 * It holds none of the simulated method's arithmetic.
 */
#ifndef DTBGEN_H
#define DTBGEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Voxel-level tables (see netgen_core.h for the exact draws). */
typedef struct dg_net dg_net;

/* Host: pull form (connection tables of section V.D) of postsynaptic
 * neurons [i0, i1): pre, cls, wbin are [(i1 - i0) * K].  Returns 0 or -1. */
int dg_host_pull(const dg_net* g, int64_t i0, int64_t i1, int32_t* pre, uint8_t* cls, uint16_t* wbin);

/* Host: outgoing CSR of a pull form by a stable counting sort; word =
 * target | class << 30.  Returns 0, -1 (bad input) or -2 (no memory). */
int dg_host_transpose(int64_t n, int32_t K, const int32_t* pre, const uint8_t* cls, const uint16_t* wbin,
                      int64_t* row_ptr, uint32_t* word, uint16_t* wbin_out);

/* Device: outgoing CSR of the whole network built in device memory; g holds
 * device pointers; d_w receives d_wtable[wbin] (w_bytes = 1, 2 or 4); d_cnt and
 * d_fill are uint32 [n] scratch.  Returns 0 or a cudaError_t value. */
int dg_dev_build(const dg_net* g, int64_t* d_row_ptr, uint32_t* d_word, void* d_w, const void* d_wtable,
                 int w_bytes, uint32_t* d_cnt, uint32_t* d_fill, void* stream);

/* Device: int8 weights with one power-of-two scale per row, from int32 weights
 * (w ~= q8 << row_shift; the shift is the smallest that keeps |q8| <= 127,
 * halves rounded away from zero).  Input preparation for the 8-bit weight
 * variant; returns 0 or a cudaError_t value. */
int dg_dev_quantize_int8(const int64_t* d_row_ptr, const int32_t* d_w32, int64_t n, int8_t* d_q8,
                         uint8_t* d_row_shift, void* stream);

#ifdef __cplusplus
}
#endif
#endif
