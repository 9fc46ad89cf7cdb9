// aes_bitslice_sbox.cuh -- GENERATED by gen_bitslice_sbox.py; do not edit by hand.
//
// Bitsliced AES S-box and inverse S-box: eight 32-bit planes in place, plane i holds bit i of
// one state byte for 32 blocks.  Derived from the field definition (GF(2^8) inverse followed
// by the affine map of App. A2; the inverse map of App. A5 followed by the inverse) through a
// normal-basis tower GF(((2^2)^2)^2) with 27 AND gates in the two outer products, mapped onto
// three-input LOP3 instructions by an exact cover; checked by the generator on all 256 inputs.
//   S-box:          77 LOP3 (117 two-input gates before mapping), N = W^2, L = 0x8, GF(16) inverse as table (tower 104, seed 1010092)
//   inverse S-box:  77 LOP3 (125 two-input gates before mapping), N = W, L = 0xE, GF(16) inverse as table (tower 14, seed 2001365)
// No memory access, no branch: the circuit's time does not depend on data or key.
// Each statement is one three-input table AES_SBOX_T(immediate, a, b, c, expression): on the
// device one lop3 instruction with the table as its immediate, on the host (the CPU test of
// the rounds) the same table as a C expression.  Left as C expressions on the device, the
// compiler regrouped the tables inside the rolled round loop (84-87 instructions per S-box).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define AES_SBOX_FN __host__ __device__ __forceinline__
#else
#define AES_SBOX_FN inline
#endif
#if defined(__CUDA_ARCH__)
template <uint32_t L>
__device__ __forceinline__ uint32_t aes_lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(L));
  return d;
}
#define AES_SBOX_T(L, a, b, c, e) aes_lop3<L>(a, b, c)
#else
#define AES_SBOX_T(L, a, b, c, e) (e)
#endif

namespace aesgb {
namespace bs {

AES_SBOX_FN void sbox_planes(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint32_t& x4, uint32_t& x5, uint32_t& x6, uint32_t& x7) {
  const uint32_t i0 = x0;
  const uint32_t i1 = x1;
  const uint32_t i2 = x2;
  const uint32_t i3 = x3;
  const uint32_t i4 = x4;
  const uint32_t i5 = x5;
  const uint32_t i6 = x6;
  const uint32_t i7 = x7;
  const uint32_t t9 = AES_SBOX_T(0x3C, i2, i7, i2, i2 ^ i7);
  const uint32_t t10 = AES_SBOX_T(0x3C, i4, i7, i4, i4 ^ i7);
  const uint32_t t11 = AES_SBOX_T(0x3C, i2, i4, i2, i2 ^ i4);
  const uint32_t t12 = AES_SBOX_T(0x96, i1, i7, t11, i1 ^ (i7 ^ t11));
  const uint32_t t14 = AES_SBOX_T(0x96, i2, i3, t12, i2 ^ (i3 ^ t12));
  const uint32_t t16 = AES_SBOX_T(0x96, i3, i6, t12, i3 ^ (i6 ^ t12));
  const uint32_t t17 = AES_SBOX_T(0x96, i4, i7, t16, i4 ^ (i7 ^ t16));
  const uint32_t t18 = AES_SBOX_T(0x96, i0, t10, t16, i0 ^ (t10 ^ t16));
  const uint32_t t20 = AES_SBOX_T(0x96, i5, i6, t17, i5 ^ (i6 ^ t17));
  const uint32_t t21 = AES_SBOX_T(0x96, i1, i7, t20, i1 ^ (i7 ^ t20));
  const uint32_t t22 = AES_SBOX_T(0x3C, i1, t21, i1, i1 ^ t21);
  const uint32_t t25 = AES_SBOX_T(0x96, i0, i5, i6, i0 ^ (i5 ^ i6));
  const uint32_t t27 = AES_SBOX_T(0x96, i1, t9, t25, i1 ^ (t9 ^ t25));
  const uint32_t t29 = AES_SBOX_T(0x96, i5, i6, t14, i5 ^ (i6 ^ t14));
  const uint32_t t31 = AES_SBOX_T(0x28, i1, i7, t20, t20 & (i1 ^ i7));
  const uint32_t t35 = AES_SBOX_T(0xA6, i1, t25, t31, i1 ^ (t31 ^ (i1 | t25)));
  const uint32_t t37 = AES_SBOX_T(0x60, i0, i4, t25, i0 & (i4 ^ t25));
  const uint32_t t38 = AES_SBOX_T(0x6A, t12, t14, t37, t37 ^ (t12 & t14));
  const uint32_t t39 = AES_SBOX_T(0x28, i0, t14, t27, t27 & (i0 ^ t14));
  const uint32_t t40 = AES_SBOX_T(0x6A, t12, t14, t39, t39 ^ (t12 & t14));
  const uint32_t t41 = AES_SBOX_T(0x60, t11, t14, t20, t11 & (t14 ^ t20));
  const uint32_t t43 = AES_SBOX_T(0x6A, t10, t17, t41, t41 ^ (t10 & t17));
  const uint32_t t45 = AES_SBOX_T(0x6A, t9, t29, t41, t41 ^ (t9 & t29));
  const uint32_t t48 = AES_SBOX_T(0x96, t16, t40, t43, t16 ^ (t40 ^ t43));
  const uint32_t t49 = AES_SBOX_T(0x56, t18, t22, t31, t31 ^ (t18 | t22));
  const uint32_t t50 = AES_SBOX_T(0x96, t43, t45, t49, t43 ^ (t45 ^ t49));
  const uint32_t t52 = AES_SBOX_T(0x96, t21, t35, t43, t21 ^ (t35 ^ t43));
  const uint32_t t53 = AES_SBOX_T(0x96, t38, t43, t45, t38 ^ (t43 ^ t45));
  const uint32_t t54 = AES_SBOX_T(0x96, t9, t29, t53, t9 ^ (t29 ^ t53));
  const uint32_t t55 = AES_SBOX_T(0xCC, t48, t50, t54, t50);
  const uint32_t t56 = AES_SBOX_T(0xE1, t48, t50, t54, ~((t48 ^ (t50 | t54))));
  const uint32_t t57 = AES_SBOX_T(0xAC, t52, t55, t56, t55 ^ (t52 & (t55 ^ t56)));
  const uint32_t t58 = AES_SBOX_T(0xD8, t50, t52, t54, t50 ^ (t54 & (t50 ^ t52)));
  const uint32_t t59 = AES_SBOX_T(0xD4, t50, t52, t54, t50 ^ ((t50 ^ t52) & (t52 ^ t54)));
  const uint32_t t60 = AES_SBOX_T(0xAC, t48, t58, t59, t58 ^ (t48 & (t58 ^ t59)));
  const uint32_t t61 = AES_SBOX_T(0xAA, t50, t52, t54, t54);
  const uint32_t t62 = AES_SBOX_T(0xC9, t50, t52, t54, ~((t52 ^ (t50 | t54))));
  const uint32_t t63 = AES_SBOX_T(0xAC, t48, t61, t62, t61 ^ (t48 & (t61 ^ t62)));
  const uint32_t t64 = AES_SBOX_T(0x0A, t50, t52, t54, t50 ^ (t50 | t54));
  const uint32_t t65 = AES_SBOX_T(0xBE, t50, t52, t54, t54 | (t50 ^ t52));
  const uint32_t t66 = AES_SBOX_T(0xAC, t48, t64, t65, t64 ^ (t48 & (t64 ^ t65)));
  const uint32_t t67 = AES_SBOX_T(0x3C, t63, t66, t63, t63 ^ t66);
  const uint32_t t69 = AES_SBOX_T(0x3C, t60, t66, t60, t60 ^ t66);
  const uint32_t t71 = AES_SBOX_T(0x96, t57, t60, t67, t57 ^ (t60 ^ t67));
  const uint32_t t72 = AES_SBOX_T(0x60, t20, t63, t66, t20 & (t63 ^ t66));
  const uint32_t t74 = AES_SBOX_T(0x6A, t18, t66, t72, t72 ^ (t18 & t66));
  const uint32_t t76 = AES_SBOX_T(0x6A, t25, t63, t72, t72 ^ (t25 & t63));
  const uint32_t t77 = AES_SBOX_T(0x60, t14, t57, t60, t14 & (t57 ^ t60));
  const uint32_t t79 = AES_SBOX_T(0x6A, i0, t60, t77, t77 ^ (i0 & t60));
  const uint32_t t80 = AES_SBOX_T(0x28, i0, t14, t57, t57 & (i0 ^ t14));
  const uint32_t t82 = AES_SBOX_T(0x28, t14, t20, t71, t71 & (t14 ^ t20));
  const uint32_t t84 = AES_SBOX_T(0x6A, t17, t69, t82, t82 ^ (t17 & t69));
  const uint32_t t85 = AES_SBOX_T(0x60, t29, t57, t63, t29 & (t57 ^ t63));
  const uint32_t t87 = AES_SBOX_T(0x28, i1, i7, t67, t67 & (i1 ^ i7));
  const uint32_t t88 = AES_SBOX_T(0x28, t18, t22, t66, t66 & (t18 ^ t22));
  const uint32_t t90 = AES_SBOX_T(0x28, i1, t25, t63, t63 & (i1 ^ t25));
  const uint32_t t92 = AES_SBOX_T(0x60, t12, t57, t60, t12 & (t57 ^ t60));
  const uint32_t t93 = AES_SBOX_T(0x28, i4, t25, t60, t60 & (i4 ^ t25));
  const uint32_t t94 = AES_SBOX_T(0x3C, t92, t93, t92, t92 ^ t93);
  const uint32_t t96 = AES_SBOX_T(0x6A, t27, t57, t92, t92 ^ (t27 & t57));
  const uint32_t t97 = AES_SBOX_T(0x28, i2, i4, t71, t71 & (i2 ^ i4));
  const uint32_t t99 = AES_SBOX_T(0x6A, t10, t69, t97, t97 ^ (t10 & t69));
  const uint32_t t100 = AES_SBOX_T(0x60, t9, t57, t63, t9 & (t57 ^ t63));
  const uint32_t t103 = AES_SBOX_T(0x96, t76, t96, t99, t76 ^ (t96 ^ t99));
  const uint32_t t104 = AES_SBOX_T(0x96, t77, t80, t103, t77 ^ (t80 ^ t103));
  const uint32_t t105 = AES_SBOX_T(0x3C, t84, t103, t84, t84 ^ t103);
  const uint32_t t107 = AES_SBOX_T(0x96, t74, t79, t104, t74 ^ (t79 ^ t104));
  const uint32_t t108 = AES_SBOX_T(0x96, t87, t90, t99, t87 ^ (t90 ^ t99));
  const uint32_t t109 = AES_SBOX_T(0x96, t74, t79, t108, t74 ^ (t79 ^ t108));
  const uint32_t t110 = AES_SBOX_T(0x96, t79, t82, t85, t79 ^ (t82 ^ t85));
  const uint32_t t111 = AES_SBOX_T(0x96, t87, t88, t110, t87 ^ (t88 ^ t110));
  const uint32_t t117 = AES_SBOX_T(0x96, t94, t103, t111, t94 ^ (t103 ^ t111));
  const uint32_t t118 = AES_SBOX_T(0x96, t84, t97, t100, t84 ^ (t97 ^ t100));
  const uint32_t t121 = AES_SBOX_T(0x0F, t109, t109, t109, ~t109);
  const uint32_t t122 = AES_SBOX_T(0x69, t76, t109, t110, ~((t76 ^ (t109 ^ t110))));
  const uint32_t t123 = AES_SBOX_T(0x69, t99, t111, t118, ~((t99 ^ (t111 ^ t118))));
  const uint32_t t124 = AES_SBOX_T(0x69, t76, t84, t104, ~((t76 ^ (t84 ^ t104))));
  x0 = t121;
  x1 = t122;
  x2 = t117;
  x3 = t107;
  x4 = t104;
  x5 = t123;
  x6 = t124;
  x7 = t105;
}

AES_SBOX_FN void inv_sbox_planes(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint32_t& x4, uint32_t& x5, uint32_t& x6, uint32_t& x7) {
  const uint32_t i0 = x0;
  const uint32_t i1 = x1;
  const uint32_t i2 = x2;
  const uint32_t i3 = x3;
  const uint32_t i4 = x4;
  const uint32_t i5 = x5;
  const uint32_t i6 = x6;
  const uint32_t i7 = x7;
  const uint32_t t8 = AES_SBOX_T(0x3C, i1, i4, i1, i1 ^ i4);
  const uint32_t t10 = AES_SBOX_T(0x96, i0, i3, i7, i0 ^ (i3 ^ i7));
  const uint32_t t11 = AES_SBOX_T(0x3C, i2, t10, i2, i2 ^ t10);
  const uint32_t t12 = AES_SBOX_T(0x96, i2, t8, t10, i2 ^ (t8 ^ t10));
  const uint32_t t13 = AES_SBOX_T(0x3C, i7, t12, i7, i7 ^ t12);
  const uint32_t t14 = AES_SBOX_T(0x3C, i5, t10, i5, i5 ^ t10);
  const uint32_t t15 = AES_SBOX_T(0x96, i0, i3, i6, i0 ^ (i3 ^ i6));
  const uint32_t t16 = AES_SBOX_T(0x3C, t12, t15, t12, t12 ^ t15);
  const uint32_t t19 = AES_SBOX_T(0x96, i1, i5, i6, i1 ^ (i5 ^ i6));
  const uint32_t t20 = AES_SBOX_T(0x3C, i0, t19, i0, i0 ^ t19);
  const uint32_t t21 = AES_SBOX_T(0x96, t12, t15, t20, t12 ^ (t15 ^ t20));
  const uint32_t t24 = AES_SBOX_T(0x96, i2, t10, t19, i2 ^ (t10 ^ t19));
  const uint32_t t26 = AES_SBOX_T(0x96, i1, i4, t20, i1 ^ (i4 ^ t20));
  const uint32_t t27 = AES_SBOX_T(0x96, i7, t8, t24, i7 ^ (t8 ^ t24));
  const uint32_t t28 = AES_SBOX_T(0x96, i5, t19, t21, i5 ^ (t19 ^ t21));
  const uint32_t t30 = AES_SBOX_T(0x96, i0, i3, t28, i0 ^ (i3 ^ t28));
  const uint32_t t42 = AES_SBOX_T(0x0C, t8, t20, t8, t8 ^ (t8 | t20));
  const uint32_t t44 = AES_SBOX_T(0x6A, t12, t16, t42, t42 ^ (t12 & t16));
  const uint32_t t46 = AES_SBOX_T(0xA6, t11, t21, t42, t11 ^ (t42 ^ (t11 | t21)));
  const uint32_t t47 = AES_SBOX_T(0x14, t14, t20, t27, t27 ^ (t27 | (t14 ^ t20)));
  const uint32_t t49 = AES_SBOX_T(0x6A, i6, t13, t47, t47 ^ (i6 & t13));
  const uint32_t t50 = AES_SBOX_T(0x21, i5, t19, t21, ~((t19 | (i5 ^ t21))));
  const uint32_t t52 = AES_SBOX_T(0x48, i7, t14, t24, t14 & (i7 ^ t24));
  const uint32_t t54 = AES_SBOX_T(0x9A, i7, t10, t52, i7 ^ (t52 ^ (i7 & t10)));
  const uint32_t t56 = AES_SBOX_T(0xA6, i5, t24, t52, i5 ^ (t52 ^ (i5 | t24)));
  const uint32_t t59 = AES_SBOX_T(0x96, t15, t49, t56, t15 ^ (t49 ^ t56));
  const uint32_t t60 = AES_SBOX_T(0x69, t26, t47, t50, ~((t26 ^ (t47 ^ t50))));
  const uint32_t t61 = AES_SBOX_T(0x96, t54, t56, t60, t54 ^ (t56 ^ t60));
  const uint32_t t63 = AES_SBOX_T(0x69, t30, t44, t56, ~((t30 ^ (t44 ^ t56))));
  const uint32_t t64 = AES_SBOX_T(0x96, t46, t54, t56, t46 ^ (t54 ^ t56));
  const uint32_t t65 = AES_SBOX_T(0x69, t26, t28, t64, ~((t26 ^ (t28 ^ t64))));
  const uint32_t t66 = AES_SBOX_T(0xEA, t59, t63, t65, t65 | (t59 & t63));
  const uint32_t t67 = AES_SBOX_T(0x8C, t59, t63, t65, t63 & (t65 | ~t59));
  const uint32_t t68 = AES_SBOX_T(0xAC, t61, t66, t67, t66 ^ (t61 & (t66 ^ t67)));
  const uint32_t t69 = AES_SBOX_T(0xAA, t59, t61, t65, t65);
  const uint32_t t70 = AES_SBOX_T(0xE1, t59, t61, t65, ~((t59 ^ (t61 | t65))));
  const uint32_t t71 = AES_SBOX_T(0xAC, t63, t69, t70, t69 ^ (t63 & (t69 ^ t70)));
  const uint32_t t72 = AES_SBOX_T(0x60, t59, t63, t65, t59 & (t63 ^ t65));
  const uint32_t t73 = AES_SBOX_T(0xF5, t59, t63, t65, t59 | ~t65);
  const uint32_t t74 = AES_SBOX_T(0xAC, t61, t72, t73, t72 ^ (t61 & (t72 ^ t73)));
  const uint32_t t75 = AES_SBOX_T(0xF0, t61, t63, t65, t61);
  const uint32_t t76 = AES_SBOX_T(0xC9, t61, t63, t65, ~((t63 ^ (t61 | t65))));
  const uint32_t t77 = AES_SBOX_T(0xAC, t59, t75, t76, t75 ^ (t59 & (t75 ^ t76)));
  const uint32_t t79 = AES_SBOX_T(0x3C, t68, t71, t68, t68 ^ t71);
  const uint32_t t81 = AES_SBOX_T(0x3C, t68, t74, t68, t68 ^ t74);
  const uint32_t t82 = AES_SBOX_T(0x96, t74, t77, t79, t74 ^ (t77 ^ t79));
  const uint32_t t83 = AES_SBOX_T(0x06, t8, t74, t77, t8 ^ (t8 | (t74 ^ t77)));
  const uint32_t t85 = AES_SBOX_T(0x6A, t12, t77, t83, t83 ^ (t12 & t77));
  const uint32_t t87 = AES_SBOX_T(0xA6, t11, t74, t83, t11 ^ (t83 ^ (t11 | t74)));
  const uint32_t t88 = AES_SBOX_T(0x0C, t27, t79, t27, t27 ^ (t27 | t79));
  const uint32_t t90 = AES_SBOX_T(0x6A, t13, t71, t88, t88 ^ (t13 & t71));
  const uint32_t t92 = AES_SBOX_T(0xA6, t19, t68, t88, t19 ^ (t88 ^ (t19 | t68)));
  const uint32_t t93 = AES_SBOX_T(0x28, i7, t24, t82, t82 & (i7 ^ t24));
  const uint32_t t94 = AES_SBOX_T(0x60, i7, t71, t77, i7 & (t71 ^ t77));
  const uint32_t t97 = AES_SBOX_T(0x6A, t24, t81, t93, t93 ^ (t24 & t81));
  const uint32_t t98 = AES_SBOX_T(0x60, t20, t74, t77, t20 & (t74 ^ t77));
  const uint32_t t100 = AES_SBOX_T(0x6A, t16, t77, t98, t98 ^ (t16 & t77));
  const uint32_t t102 = AES_SBOX_T(0x6A, t21, t74, t98, t98 ^ (t21 & t74));
  const uint32_t t103 = AES_SBOX_T(0x28, t14, t20, t79, t79 & (t14 ^ t20));
  const uint32_t t104 = AES_SBOX_T(0x82, i6, t13, t71, t71 & ~((i6 ^ t13)));
  const uint32_t t106 = AES_SBOX_T(0x82, i5, t21, t68, t68 & ~((i5 ^ t21)));
  const uint32_t t108 = AES_SBOX_T(0xC0, t14, t82, t14, t14 & t82);
  const uint32_t t109 = AES_SBOX_T(0x06, t10, t71, t77, t10 ^ (t10 | (t71 ^ t77)));
  const uint32_t t112 = AES_SBOX_T(0xA6, i5, t81, t108, i5 ^ (t108 ^ (i5 | t81)));
  const uint32_t t114 = AES_SBOX_T(0x96, t100, t103, t104, t100 ^ (t103 ^ t104));
  const uint32_t t115 = AES_SBOX_T(0x96, t90, t92, t114, t90 ^ (t92 ^ t114));
  const uint32_t t116 = AES_SBOX_T(0x96, t93, t94, t115, t93 ^ (t94 ^ t115));
  const uint32_t t117 = AES_SBOX_T(0x96, t102, t108, t109, t102 ^ (t108 ^ t109));
  const uint32_t t118 = AES_SBOX_T(0x96, t103, t104, t117, t103 ^ (t104 ^ t117));
  const uint32_t t120 = AES_SBOX_T(0x96, t85, t87, t115, t85 ^ (t87 ^ t115));
  const uint32_t t122 = AES_SBOX_T(0x96, t97, t100, t112, t97 ^ (t100 ^ t112));
  const uint32_t t123 = AES_SBOX_T(0x3C, t85, t122, t85, t85 ^ t122);
  const uint32_t t125 = AES_SBOX_T(0x96, t112, t117, t120, t112 ^ (t117 ^ t120));
  const uint32_t t127 = AES_SBOX_T(0x96, t90, t118, t122, t90 ^ (t118 ^ t122));
  const uint32_t t128 = AES_SBOX_T(0x96, t102, t103, t106, t102 ^ (t103 ^ t106));
  const uint32_t t130 = AES_SBOX_T(0x96, t114, t116, t128, t114 ^ (t116 ^ t128));
  const uint32_t t132 = AES_SBOX_T(0x96, t120, t127, t128, t120 ^ (t127 ^ t128));
  x0 = t125;
  x1 = t123;
  x2 = t118;
  x3 = t130;
  x4 = t116;
  x5 = t132;
  x6 = t120;
  x7 = t127;
}

}  // namespace bs
}  // namespace aesgb
