// sg_mma.cuh -- warp-level BF16 tensor-core tiles for the dueling Q-network.
//
// One tile is C[16 x 8] += A[16 x 16] * B[16 x 8] (mma.sync m16n8k16, BF16
// inputs, FP32 accumulators).  Operands come from shared memory through
// ldmatrix; every matrix row starts on a 16-byte boundary and row strides are
// padded by 8 elements so that the eight rows of one 8x8 load fall in
// distinct banks.
//
// Operand storage (all row-major in shared memory, element (r, c) at
// base[r * ld + c]):
//   A "row":  A[m][k] stored as rows m        -> ldmatrix
//   A "col":  A[m][k] stored as rows k (A^T)  -> ldmatrix.trans
//   B "col":  B[k][n] stored as rows n (B^T, e.g. a weight matrix W[n][k])
//             -> ldmatrix
//   B "row":  B[k][n] stored as rows k        -> ldmatrix.trans
// Fragment ownership (PTX ISA, mma.m16n8k16): with g = lane / 4, q = lane % 4,
// C element (g, 2q..2q+1) is c[0..1] and (g + 8, 2q..2q+1) is c[2..3].
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace sg {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment of the 16x16 block at (m0, k0).
__device__ __forceinline__ void load_a_row(uint32_t (&a)[4], const bf16* A, int ld, int m0, int k0, int lane) {
  ldsm_x4(a, A + (m0 + (lane & 15)) * ld + k0 + (lane >> 4) * 8);
}
__device__ __forceinline__ void load_a_col(uint32_t (&a)[4], const bf16* At, int ld, int m0, int k0, int lane) {
  // matrices: (k0..7, m0..7), (k0..7, m0+8..15), (k0+8.., m0..), (k0+8.., m0+8..)
  const int mat = lane >> 3, r = lane & 7;
  ldsm_x4_t(a, At + (k0 + r + ((mat & 2) ? 8 : 0)) * ld + m0 + ((mat & 1) ? 8 : 0));
}
// B fragment of the 16x8 block at (k0, n0).
__device__ __forceinline__ void load_b_col(uint32_t& b0, uint32_t& b1, const bf16* Bt, int ld, int k0, int n0,
                                           int lane) {
  ldsm_x2(b0, b1, Bt + (n0 + (lane & 7)) * ld + k0 + ((lane >> 3) & 1) * 8);
}
__device__ __forceinline__ void load_b_row(uint32_t& b0, uint32_t& b1, const bf16* B, int ld, int k0, int n0,
                                           int lane) {
  ldsm_x2_t(b0, b1, B + (k0 + (lane & 7) + ((lane >> 3) & 1) * 8) * ld + n0);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
// max(lo, 0) and max(hi, 0) rounded to BF16 (nearest even) in one
// conversion: ReLU commutes with the monotone rounding, so this equals
// pack_bf16x2(fmaxf(lo, 0), fmaxf(hi, 0)) up to the sign of a zero
// (a NaN stays NaN).
__device__ __forceinline__ uint32_t pack_bf16x2_relu(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

}  // namespace sg
