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
// Each statement is one three-input table (its LOP3 immediate in the comment), written as a C
// expression; on the device an empty asm fence after each keeps the compiler from merging
// tables, so that each folds into that single instruction.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define AES_SBOX_FN __host__ __device__ __forceinline__
#else
#define AES_SBOX_FN inline
#endif
#if defined(__CUDA_ARCH__)
#define AES_SBOX_FENCE(v) asm("" : "+r"(v))
#else
#define AES_SBOX_FENCE(v) ((void)0)
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
  uint32_t t9 = i2 ^ i7;  // lop3 0x3C
  AES_SBOX_FENCE(t9);
  uint32_t t10 = i4 ^ i7;  // lop3 0x3C
  AES_SBOX_FENCE(t10);
  uint32_t t11 = i2 ^ i4;  // lop3 0x3C
  AES_SBOX_FENCE(t11);
  uint32_t t12 = i1 ^ (i7 ^ t11);  // lop3 0x96
  AES_SBOX_FENCE(t12);
  uint32_t t14 = i2 ^ (i3 ^ t12);  // lop3 0x96
  AES_SBOX_FENCE(t14);
  uint32_t t16 = i3 ^ (i6 ^ t12);  // lop3 0x96
  AES_SBOX_FENCE(t16);
  uint32_t t17 = i4 ^ (i7 ^ t16);  // lop3 0x96
  AES_SBOX_FENCE(t17);
  uint32_t t18 = i0 ^ (t10 ^ t16);  // lop3 0x96
  AES_SBOX_FENCE(t18);
  uint32_t t20 = i5 ^ (i6 ^ t17);  // lop3 0x96
  AES_SBOX_FENCE(t20);
  uint32_t t21 = i1 ^ (i7 ^ t20);  // lop3 0x96
  AES_SBOX_FENCE(t21);
  uint32_t t22 = i1 ^ t21;  // lop3 0x3C
  AES_SBOX_FENCE(t22);
  uint32_t t25 = i0 ^ (i5 ^ i6);  // lop3 0x96
  AES_SBOX_FENCE(t25);
  uint32_t t27 = i1 ^ (t9 ^ t25);  // lop3 0x96
  AES_SBOX_FENCE(t27);
  uint32_t t29 = i5 ^ (i6 ^ t14);  // lop3 0x96
  AES_SBOX_FENCE(t29);
  uint32_t t31 = t20 & (i1 ^ i7);  // lop3 0x28
  AES_SBOX_FENCE(t31);
  uint32_t t35 = i1 ^ (t31 ^ (i1 | t25));  // lop3 0xA6
  AES_SBOX_FENCE(t35);
  uint32_t t37 = i0 & (i4 ^ t25);  // lop3 0x60
  AES_SBOX_FENCE(t37);
  uint32_t t38 = t37 ^ (t12 & t14);  // lop3 0x6A
  AES_SBOX_FENCE(t38);
  uint32_t t39 = t27 & (i0 ^ t14);  // lop3 0x28
  AES_SBOX_FENCE(t39);
  uint32_t t40 = t39 ^ (t12 & t14);  // lop3 0x6A
  AES_SBOX_FENCE(t40);
  uint32_t t41 = t11 & (t14 ^ t20);  // lop3 0x60
  AES_SBOX_FENCE(t41);
  uint32_t t43 = t41 ^ (t10 & t17);  // lop3 0x6A
  AES_SBOX_FENCE(t43);
  uint32_t t45 = t41 ^ (t9 & t29);  // lop3 0x6A
  AES_SBOX_FENCE(t45);
  uint32_t t48 = t16 ^ (t40 ^ t43);  // lop3 0x96
  AES_SBOX_FENCE(t48);
  uint32_t t49 = t31 ^ (t18 | t22);  // lop3 0x56
  AES_SBOX_FENCE(t49);
  uint32_t t50 = t43 ^ (t45 ^ t49);  // lop3 0x96
  AES_SBOX_FENCE(t50);
  uint32_t t52 = t21 ^ (t35 ^ t43);  // lop3 0x96
  AES_SBOX_FENCE(t52);
  uint32_t t53 = t38 ^ (t43 ^ t45);  // lop3 0x96
  AES_SBOX_FENCE(t53);
  uint32_t t54 = t9 ^ (t29 ^ t53);  // lop3 0x96
  AES_SBOX_FENCE(t54);
  uint32_t t55 = t50;  // lop3 0xCC
  AES_SBOX_FENCE(t55);
  uint32_t t56 = ~((t48 ^ (t50 | t54)));  // lop3 0xE1
  AES_SBOX_FENCE(t56);
  uint32_t t57 = t55 ^ (t52 & (t55 ^ t56));  // lop3 0xAC
  AES_SBOX_FENCE(t57);
  uint32_t t58 = t50 ^ (t54 & (t50 ^ t52));  // lop3 0xD8
  AES_SBOX_FENCE(t58);
  uint32_t t59 = t50 ^ ((t50 ^ t52) & (t52 ^ t54));  // lop3 0xD4
  AES_SBOX_FENCE(t59);
  uint32_t t60 = t58 ^ (t48 & (t58 ^ t59));  // lop3 0xAC
  AES_SBOX_FENCE(t60);
  uint32_t t61 = t54;  // lop3 0xAA
  AES_SBOX_FENCE(t61);
  uint32_t t62 = ~((t52 ^ (t50 | t54)));  // lop3 0xC9
  AES_SBOX_FENCE(t62);
  uint32_t t63 = t61 ^ (t48 & (t61 ^ t62));  // lop3 0xAC
  AES_SBOX_FENCE(t63);
  uint32_t t64 = t50 ^ (t50 | t54);  // lop3 0x0A
  AES_SBOX_FENCE(t64);
  uint32_t t65 = t54 | (t50 ^ t52);  // lop3 0xBE
  AES_SBOX_FENCE(t65);
  uint32_t t66 = t64 ^ (t48 & (t64 ^ t65));  // lop3 0xAC
  AES_SBOX_FENCE(t66);
  uint32_t t67 = t63 ^ t66;  // lop3 0x3C
  AES_SBOX_FENCE(t67);
  uint32_t t69 = t60 ^ t66;  // lop3 0x3C
  AES_SBOX_FENCE(t69);
  uint32_t t71 = t57 ^ (t60 ^ t67);  // lop3 0x96
  AES_SBOX_FENCE(t71);
  uint32_t t72 = t20 & (t63 ^ t66);  // lop3 0x60
  AES_SBOX_FENCE(t72);
  uint32_t t74 = t72 ^ (t18 & t66);  // lop3 0x6A
  AES_SBOX_FENCE(t74);
  uint32_t t76 = t72 ^ (t25 & t63);  // lop3 0x6A
  AES_SBOX_FENCE(t76);
  uint32_t t77 = t14 & (t57 ^ t60);  // lop3 0x60
  AES_SBOX_FENCE(t77);
  uint32_t t79 = t77 ^ (i0 & t60);  // lop3 0x6A
  AES_SBOX_FENCE(t79);
  uint32_t t80 = t57 & (i0 ^ t14);  // lop3 0x28
  AES_SBOX_FENCE(t80);
  uint32_t t82 = t71 & (t14 ^ t20);  // lop3 0x28
  AES_SBOX_FENCE(t82);
  uint32_t t84 = t82 ^ (t17 & t69);  // lop3 0x6A
  AES_SBOX_FENCE(t84);
  uint32_t t85 = t29 & (t57 ^ t63);  // lop3 0x60
  AES_SBOX_FENCE(t85);
  uint32_t t87 = t67 & (i1 ^ i7);  // lop3 0x28
  AES_SBOX_FENCE(t87);
  uint32_t t88 = t66 & (t18 ^ t22);  // lop3 0x28
  AES_SBOX_FENCE(t88);
  uint32_t t90 = t63 & (i1 ^ t25);  // lop3 0x28
  AES_SBOX_FENCE(t90);
  uint32_t t92 = t12 & (t57 ^ t60);  // lop3 0x60
  AES_SBOX_FENCE(t92);
  uint32_t t93 = t60 & (i4 ^ t25);  // lop3 0x28
  AES_SBOX_FENCE(t93);
  uint32_t t94 = t92 ^ t93;  // lop3 0x3C
  AES_SBOX_FENCE(t94);
  uint32_t t96 = t92 ^ (t27 & t57);  // lop3 0x6A
  AES_SBOX_FENCE(t96);
  uint32_t t97 = t71 & (i2 ^ i4);  // lop3 0x28
  AES_SBOX_FENCE(t97);
  uint32_t t99 = t97 ^ (t10 & t69);  // lop3 0x6A
  AES_SBOX_FENCE(t99);
  uint32_t t100 = t9 & (t57 ^ t63);  // lop3 0x60
  AES_SBOX_FENCE(t100);
  uint32_t t103 = t76 ^ (t96 ^ t99);  // lop3 0x96
  AES_SBOX_FENCE(t103);
  uint32_t t104 = t77 ^ (t80 ^ t103);  // lop3 0x96
  AES_SBOX_FENCE(t104);
  uint32_t t105 = t84 ^ t103;  // lop3 0x3C
  AES_SBOX_FENCE(t105);
  uint32_t t107 = t74 ^ (t79 ^ t104);  // lop3 0x96
  AES_SBOX_FENCE(t107);
  uint32_t t108 = t87 ^ (t90 ^ t99);  // lop3 0x96
  AES_SBOX_FENCE(t108);
  uint32_t t109 = t74 ^ (t79 ^ t108);  // lop3 0x96
  AES_SBOX_FENCE(t109);
  uint32_t t110 = t79 ^ (t82 ^ t85);  // lop3 0x96
  AES_SBOX_FENCE(t110);
  uint32_t t111 = t87 ^ (t88 ^ t110);  // lop3 0x96
  AES_SBOX_FENCE(t111);
  uint32_t t117 = t94 ^ (t103 ^ t111);  // lop3 0x96
  AES_SBOX_FENCE(t117);
  uint32_t t118 = t84 ^ (t97 ^ t100);  // lop3 0x96
  AES_SBOX_FENCE(t118);
  uint32_t t121 = ~t109;  // lop3 0x0F
  AES_SBOX_FENCE(t121);
  uint32_t t122 = ~((t76 ^ (t109 ^ t110)));  // lop3 0x69
  AES_SBOX_FENCE(t122);
  uint32_t t123 = ~((t99 ^ (t111 ^ t118)));  // lop3 0x69
  AES_SBOX_FENCE(t123);
  uint32_t t124 = ~((t76 ^ (t84 ^ t104)));  // lop3 0x69
  AES_SBOX_FENCE(t124);
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
  uint32_t t8 = i1 ^ i4;  // lop3 0x3C
  AES_SBOX_FENCE(t8);
  uint32_t t10 = i0 ^ (i3 ^ i7);  // lop3 0x96
  AES_SBOX_FENCE(t10);
  uint32_t t11 = i2 ^ t10;  // lop3 0x3C
  AES_SBOX_FENCE(t11);
  uint32_t t12 = i2 ^ (t8 ^ t10);  // lop3 0x96
  AES_SBOX_FENCE(t12);
  uint32_t t13 = i7 ^ t12;  // lop3 0x3C
  AES_SBOX_FENCE(t13);
  uint32_t t14 = i5 ^ t10;  // lop3 0x3C
  AES_SBOX_FENCE(t14);
  uint32_t t15 = i0 ^ (i3 ^ i6);  // lop3 0x96
  AES_SBOX_FENCE(t15);
  uint32_t t16 = t12 ^ t15;  // lop3 0x3C
  AES_SBOX_FENCE(t16);
  uint32_t t19 = i1 ^ (i5 ^ i6);  // lop3 0x96
  AES_SBOX_FENCE(t19);
  uint32_t t20 = i0 ^ t19;  // lop3 0x3C
  AES_SBOX_FENCE(t20);
  uint32_t t21 = t12 ^ (t15 ^ t20);  // lop3 0x96
  AES_SBOX_FENCE(t21);
  uint32_t t24 = i2 ^ (t10 ^ t19);  // lop3 0x96
  AES_SBOX_FENCE(t24);
  uint32_t t26 = i1 ^ (i4 ^ t20);  // lop3 0x96
  AES_SBOX_FENCE(t26);
  uint32_t t27 = i7 ^ (t8 ^ t24);  // lop3 0x96
  AES_SBOX_FENCE(t27);
  uint32_t t28 = i5 ^ (t19 ^ t21);  // lop3 0x96
  AES_SBOX_FENCE(t28);
  uint32_t t30 = i0 ^ (i3 ^ t28);  // lop3 0x96
  AES_SBOX_FENCE(t30);
  uint32_t t42 = t8 ^ (t8 | t20);  // lop3 0x0C
  AES_SBOX_FENCE(t42);
  uint32_t t44 = t42 ^ (t12 & t16);  // lop3 0x6A
  AES_SBOX_FENCE(t44);
  uint32_t t46 = t11 ^ (t42 ^ (t11 | t21));  // lop3 0xA6
  AES_SBOX_FENCE(t46);
  uint32_t t47 = t27 ^ (t27 | (t14 ^ t20));  // lop3 0x14
  AES_SBOX_FENCE(t47);
  uint32_t t49 = t47 ^ (i6 & t13);  // lop3 0x6A
  AES_SBOX_FENCE(t49);
  uint32_t t50 = ~((t19 | (i5 ^ t21)));  // lop3 0x21
  AES_SBOX_FENCE(t50);
  uint32_t t52 = t14 & (i7 ^ t24);  // lop3 0x48
  AES_SBOX_FENCE(t52);
  uint32_t t54 = i7 ^ (t52 ^ (i7 & t10));  // lop3 0x9A
  AES_SBOX_FENCE(t54);
  uint32_t t56 = i5 ^ (t52 ^ (i5 | t24));  // lop3 0xA6
  AES_SBOX_FENCE(t56);
  uint32_t t59 = t15 ^ (t49 ^ t56);  // lop3 0x96
  AES_SBOX_FENCE(t59);
  uint32_t t60 = ~((t26 ^ (t47 ^ t50)));  // lop3 0x69
  AES_SBOX_FENCE(t60);
  uint32_t t61 = t54 ^ (t56 ^ t60);  // lop3 0x96
  AES_SBOX_FENCE(t61);
  uint32_t t63 = ~((t30 ^ (t44 ^ t56)));  // lop3 0x69
  AES_SBOX_FENCE(t63);
  uint32_t t64 = t46 ^ (t54 ^ t56);  // lop3 0x96
  AES_SBOX_FENCE(t64);
  uint32_t t65 = ~((t26 ^ (t28 ^ t64)));  // lop3 0x69
  AES_SBOX_FENCE(t65);
  uint32_t t66 = t65 | (t59 & t63);  // lop3 0xEA
  AES_SBOX_FENCE(t66);
  uint32_t t67 = t63 & (t65 | ~t59);  // lop3 0x8C
  AES_SBOX_FENCE(t67);
  uint32_t t68 = t66 ^ (t61 & (t66 ^ t67));  // lop3 0xAC
  AES_SBOX_FENCE(t68);
  uint32_t t69 = t65;  // lop3 0xAA
  AES_SBOX_FENCE(t69);
  uint32_t t70 = ~((t59 ^ (t61 | t65)));  // lop3 0xE1
  AES_SBOX_FENCE(t70);
  uint32_t t71 = t69 ^ (t63 & (t69 ^ t70));  // lop3 0xAC
  AES_SBOX_FENCE(t71);
  uint32_t t72 = t59 & (t63 ^ t65);  // lop3 0x60
  AES_SBOX_FENCE(t72);
  uint32_t t73 = t59 | ~t65;  // lop3 0xF5
  AES_SBOX_FENCE(t73);
  uint32_t t74 = t72 ^ (t61 & (t72 ^ t73));  // lop3 0xAC
  AES_SBOX_FENCE(t74);
  uint32_t t75 = t61;  // lop3 0xF0
  AES_SBOX_FENCE(t75);
  uint32_t t76 = ~((t63 ^ (t61 | t65)));  // lop3 0xC9
  AES_SBOX_FENCE(t76);
  uint32_t t77 = t75 ^ (t59 & (t75 ^ t76));  // lop3 0xAC
  AES_SBOX_FENCE(t77);
  uint32_t t79 = t68 ^ t71;  // lop3 0x3C
  AES_SBOX_FENCE(t79);
  uint32_t t81 = t68 ^ t74;  // lop3 0x3C
  AES_SBOX_FENCE(t81);
  uint32_t t82 = t74 ^ (t77 ^ t79);  // lop3 0x96
  AES_SBOX_FENCE(t82);
  uint32_t t83 = t8 ^ (t8 | (t74 ^ t77));  // lop3 0x06
  AES_SBOX_FENCE(t83);
  uint32_t t85 = t83 ^ (t12 & t77);  // lop3 0x6A
  AES_SBOX_FENCE(t85);
  uint32_t t87 = t11 ^ (t83 ^ (t11 | t74));  // lop3 0xA6
  AES_SBOX_FENCE(t87);
  uint32_t t88 = t27 ^ (t27 | t79);  // lop3 0x0C
  AES_SBOX_FENCE(t88);
  uint32_t t90 = t88 ^ (t13 & t71);  // lop3 0x6A
  AES_SBOX_FENCE(t90);
  uint32_t t92 = t19 ^ (t88 ^ (t19 | t68));  // lop3 0xA6
  AES_SBOX_FENCE(t92);
  uint32_t t93 = t82 & (i7 ^ t24);  // lop3 0x28
  AES_SBOX_FENCE(t93);
  uint32_t t94 = i7 & (t71 ^ t77);  // lop3 0x60
  AES_SBOX_FENCE(t94);
  uint32_t t97 = t93 ^ (t24 & t81);  // lop3 0x6A
  AES_SBOX_FENCE(t97);
  uint32_t t98 = t20 & (t74 ^ t77);  // lop3 0x60
  AES_SBOX_FENCE(t98);
  uint32_t t100 = t98 ^ (t16 & t77);  // lop3 0x6A
  AES_SBOX_FENCE(t100);
  uint32_t t102 = t98 ^ (t21 & t74);  // lop3 0x6A
  AES_SBOX_FENCE(t102);
  uint32_t t103 = t79 & (t14 ^ t20);  // lop3 0x28
  AES_SBOX_FENCE(t103);
  uint32_t t104 = t71 & ~((i6 ^ t13));  // lop3 0x82
  AES_SBOX_FENCE(t104);
  uint32_t t106 = t68 & ~((i5 ^ t21));  // lop3 0x82
  AES_SBOX_FENCE(t106);
  uint32_t t108 = t14 & t82;  // lop3 0xC0
  AES_SBOX_FENCE(t108);
  uint32_t t109 = t10 ^ (t10 | (t71 ^ t77));  // lop3 0x06
  AES_SBOX_FENCE(t109);
  uint32_t t112 = i5 ^ (t108 ^ (i5 | t81));  // lop3 0xA6
  AES_SBOX_FENCE(t112);
  uint32_t t114 = t100 ^ (t103 ^ t104);  // lop3 0x96
  AES_SBOX_FENCE(t114);
  uint32_t t115 = t90 ^ (t92 ^ t114);  // lop3 0x96
  AES_SBOX_FENCE(t115);
  uint32_t t116 = t93 ^ (t94 ^ t115);  // lop3 0x96
  AES_SBOX_FENCE(t116);
  uint32_t t117 = t102 ^ (t108 ^ t109);  // lop3 0x96
  AES_SBOX_FENCE(t117);
  uint32_t t118 = t103 ^ (t104 ^ t117);  // lop3 0x96
  AES_SBOX_FENCE(t118);
  uint32_t t120 = t85 ^ (t87 ^ t115);  // lop3 0x96
  AES_SBOX_FENCE(t120);
  uint32_t t122 = t97 ^ (t100 ^ t112);  // lop3 0x96
  AES_SBOX_FENCE(t122);
  uint32_t t123 = t85 ^ t122;  // lop3 0x3C
  AES_SBOX_FENCE(t123);
  uint32_t t125 = t112 ^ (t117 ^ t120);  // lop3 0x96
  AES_SBOX_FENCE(t125);
  uint32_t t127 = t90 ^ (t118 ^ t122);  // lop3 0x96
  AES_SBOX_FENCE(t127);
  uint32_t t128 = t102 ^ (t103 ^ t106);  // lop3 0x96
  AES_SBOX_FENCE(t128);
  uint32_t t130 = t114 ^ (t116 ^ t128);  // lop3 0x96
  AES_SBOX_FENCE(t130);
  uint32_t t132 = t120 ^ (t127 ^ t128);  // lop3 0x96
  AES_SBOX_FENCE(t132);
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
