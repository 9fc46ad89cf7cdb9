// aes_bitslice_sbox.cuh -- GENERATED by gen_bitslice_sbox.py; do not edit by hand.
//
// Bitsliced AES S-box and inverse S-box: eight 32-bit planes in place, plane i holds bit i of
// one state byte for 32 blocks.  Derived from the field definition (GF(2^8) inverse followed
// by the affine map of App. A2; the inverse map of App. A5 followed by the inverse) through
// the tower GF((2^4)^2); checked by the generator on all 256 inputs.
//   S-box tower:      zeta = 0xE1 (root of z^4+z+1), lambda = 0xA, eta = 0x42; linear-layer XORs = 34
//   inverse tower:    zeta = 0xE1, lambda = 0xD, eta = 0x1E; linear-layer XORs = 35
// Every memory access is absent: the circuit's time does not depend on data or key.
#pragma once
#include <cstdint>

namespace aesgb {
namespace bs {

template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

__device__ __forceinline__ void sbox_planes(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint32_t& x4, uint32_t& x5, uint32_t& x6, uint32_t& x7) {
  const uint32_t t1 = x4 ^ x5;
  const uint32_t t2 = x3 ^ x6;
  const uint32_t t3 = x7 ^ t2;
  const uint32_t t4 = x0 ^ t1;
  const uint32_t t5 = x1 ^ x6;
  const uint32_t t6 = x2 ^ x3;
  const uint32_t t7 = x2 ^ t3;
  const uint32_t t8 = x5 ^ x7;
  const uint32_t t9 = x7 ^ t1;
  const uint32_t t10 = x0 ^ x5;
  const uint32_t t11 = x5 ^ t6;
  const uint32_t t12 = x7 ^ t5;
  const uint32_t t13 = x1 ^ t3;
  const uint32_t t14 = x4 ^ t7;
  const uint32_t t15 = t6 ^ t8;
  const uint32_t t16 = t1 ^ t5;
  const uint32_t t17 = t8;
  const uint32_t t18 = t4 ^ t7;
  const uint32_t t19 = x7;
  const uint32_t t20 = t9;
  const uint32_t t21 = x1 ^ x5 ^ t2;
  const uint32_t t22 = t4;
  const uint32_t t23 = x1 ^ t9;
  const uint32_t t24 = x3 ^ t1;
  const uint32_t t25 = t3;
  const uint32_t t26 = (t15 & t13) ^ (t16 & t12) ^ (t17 & t11);
  const uint32_t t27 = (t16 & t13) ^ (t17 & t12);
  const uint32_t t28 = (t17 & t13);
  const uint32_t t29 = (t14 & t10) ^ t26;
  const uint32_t t30 = (t14 & t11) ^ (t15 & t10) ^ t26 ^ t27;
  const uint32_t t31 = (t14 & t12) ^ (t15 & t11) ^ (t16 & t10) ^ t27 ^ t28;
  const uint32_t t32 = (t14 & t13) ^ (t15 & t12) ^ (t16 & t11) ^ (t17 & t10) ^ t28;
  const uint32_t t33 = t22 ^ t29;
  const uint32_t t34 = t23 ^ t30;
  const uint32_t t35 = t24 ^ t31;
  const uint32_t t36 = t25 ^ t32;
  const uint32_t t37 = lop3<0x3E>(t33, t34, t35);
  const uint32_t t38 = lop3<0x49>(t33, t34, t35);
  const uint32_t t39 = lop3<0xCA>(t36, t38, t37);  // d3 ? f1 : f0
  const uint32_t t40 = lop3<0xE8>(t33, t34, t35);
  const uint32_t t41 = lop3<0x1B>(t33, t34, t35);
  const uint32_t t42 = lop3<0xCA>(t36, t41, t40);  // d3 ? f1 : f0
  const uint32_t t43 = lop3<0xCA>(t33, t34, t35);
  const uint32_t t44 = lop3<0x65>(t33, t34, t35);
  const uint32_t t45 = lop3<0xCA>(t36, t44, t43);  // d3 ? f1 : f0
  const uint32_t t46 = lop3<0x66>(t33, t34, t35);
  const uint32_t t47 = lop3<0x87>(t33, t34, t35);
  const uint32_t t48 = lop3<0xCA>(t36, t47, t46);  // d3 ? f1 : f0
  const uint32_t t49 = (t15 & t48) ^ (t16 & t45) ^ (t17 & t42);
  const uint32_t t50 = (t16 & t48) ^ (t17 & t45);
  const uint32_t t51 = (t17 & t48);
  const uint32_t t52 = (t14 & t39) ^ t49;
  const uint32_t t53 = (t14 & t42) ^ (t15 & t39) ^ t49 ^ t50;
  const uint32_t t54 = (t14 & t45) ^ (t15 & t42) ^ (t16 & t39) ^ t50 ^ t51;
  const uint32_t t55 = (t14 & t48) ^ (t15 & t45) ^ (t16 & t42) ^ (t17 & t39) ^ t51;
  const uint32_t t56 = (t19 & t48) ^ (t20 & t45) ^ (t21 & t42);
  const uint32_t t57 = (t20 & t48) ^ (t21 & t45);
  const uint32_t t58 = (t21 & t48);
  const uint32_t t59 = (t18 & t39) ^ t56;
  const uint32_t t60 = (t18 & t42) ^ (t19 & t39) ^ t56 ^ t57;
  const uint32_t t61 = (t18 & t45) ^ (t19 & t42) ^ (t20 & t39) ^ t57 ^ t58;
  const uint32_t t62 = (t18 & t48) ^ (t19 & t45) ^ (t20 & t42) ^ (t21 & t39) ^ t58;
  const uint32_t t63 = t52 ^ t55;
  const uint32_t t64 = t60 ^ t61;
  const uint32_t t65 = t53 ^ t63;
  const uint32_t t66 = t59 ^ t65;
  const uint32_t t67 = ~(t66);
  const uint32_t t68 = ~(t59 ^ t61);
  const uint32_t t69 = t59 ^ t60 ^ t62;
  const uint32_t t70 = t59 ^ t52 ^ t54;
  const uint32_t t71 = t64 ^ t66;
  const uint32_t t72 = ~(t64 ^ t65);
  const uint32_t t73 = ~(t63);
  const uint32_t t74 = t62 ^ t52 ^ t64;
  x0 = t67;
  x1 = t68;
  x2 = t69;
  x3 = t70;
  x4 = t71;
  x5 = t72;
  x6 = t73;
  x7 = t74;
}

__device__ __forceinline__ void inv_sbox_planes(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint32_t& x4, uint32_t& x5, uint32_t& x6, uint32_t& x7) {
  const uint32_t t1 = x2 ^ x7;
  const uint32_t t2 = x1 ^ x3;
  const uint32_t t3 = x4 ^ x5;
  const uint32_t t4 = x0 ^ x6;
  const uint32_t t5 = x1 ^ x6;
  const uint32_t t6 = x3 ^ t1;
  const uint32_t t7 = x5 ^ x7;
  const uint32_t t8 = t1 ^ t2;
  const uint32_t t9 = ~(t8);
  const uint32_t t10 = ~(x4 ^ t2 ^ t4);
  const uint32_t t11 = ~(t3 ^ t5);
  const uint32_t t12 = ~(x2 ^ x5 ^ t5);
  const uint32_t t13 = ~(x1 ^ t1);
  const uint32_t t14 = ~(t3 ^ t4);
  const uint32_t t15 = t3 ^ t8;
  const uint32_t t16 = t1 ^ t5;
  const uint32_t t17 = x3;
  const uint32_t t18 = x5 ^ t2;
  const uint32_t t19 = ~(x6 ^ t6);
  const uint32_t t20 = ~(t7);
  const uint32_t t21 = t4 ^ t6;
  const uint32_t t22 = ~(t1 ^ t3);
  const uint32_t t23 = ~(x0 ^ x2);
  const uint32_t t24 = x6 ^ t7;
  const uint32_t t25 = (t14 & t12) ^ (t15 & t11) ^ (t16 & t10);
  const uint32_t t26 = (t15 & t12) ^ (t16 & t11);
  const uint32_t t27 = (t16 & t12);
  const uint32_t t28 = (t13 & t9) ^ t25;
  const uint32_t t29 = (t13 & t10) ^ (t14 & t9) ^ t25 ^ t26;
  const uint32_t t30 = (t13 & t11) ^ (t14 & t10) ^ (t15 & t9) ^ t26 ^ t27;
  const uint32_t t31 = (t13 & t12) ^ (t14 & t11) ^ (t15 & t10) ^ (t16 & t9) ^ t27;
  const uint32_t t32 = t21 ^ t28;
  const uint32_t t33 = t22 ^ t29;
  const uint32_t t34 = t23 ^ t30;
  const uint32_t t35 = t24 ^ t31;
  const uint32_t t36 = lop3<0x3E>(t32, t33, t34);
  const uint32_t t37 = lop3<0x49>(t32, t33, t34);
  const uint32_t t38 = lop3<0xCA>(t35, t37, t36);  // d3 ? f1 : f0
  const uint32_t t39 = lop3<0xE8>(t32, t33, t34);
  const uint32_t t40 = lop3<0x1B>(t32, t33, t34);
  const uint32_t t41 = lop3<0xCA>(t35, t40, t39);  // d3 ? f1 : f0
  const uint32_t t42 = lop3<0xCA>(t32, t33, t34);
  const uint32_t t43 = lop3<0x65>(t32, t33, t34);
  const uint32_t t44 = lop3<0xCA>(t35, t43, t42);  // d3 ? f1 : f0
  const uint32_t t45 = lop3<0x66>(t32, t33, t34);
  const uint32_t t46 = lop3<0x87>(t32, t33, t34);
  const uint32_t t47 = lop3<0xCA>(t35, t46, t45);  // d3 ? f1 : f0
  const uint32_t t48 = (t14 & t47) ^ (t15 & t44) ^ (t16 & t41);
  const uint32_t t49 = (t15 & t47) ^ (t16 & t44);
  const uint32_t t50 = (t16 & t47);
  const uint32_t t51 = (t13 & t38) ^ t48;
  const uint32_t t52 = (t13 & t41) ^ (t14 & t38) ^ t48 ^ t49;
  const uint32_t t53 = (t13 & t44) ^ (t14 & t41) ^ (t15 & t38) ^ t49 ^ t50;
  const uint32_t t54 = (t13 & t47) ^ (t14 & t44) ^ (t15 & t41) ^ (t16 & t38) ^ t50;
  const uint32_t t55 = (t18 & t47) ^ (t19 & t44) ^ (t20 & t41);
  const uint32_t t56 = (t19 & t47) ^ (t20 & t44);
  const uint32_t t57 = (t20 & t47);
  const uint32_t t58 = (t17 & t38) ^ t55;
  const uint32_t t59 = (t17 & t41) ^ (t18 & t38) ^ t55 ^ t56;
  const uint32_t t60 = (t17 & t44) ^ (t18 & t41) ^ (t19 & t38) ^ t56 ^ t57;
  const uint32_t t61 = (t17 & t47) ^ (t18 & t44) ^ (t19 & t41) ^ (t20 & t38) ^ t57;
  const uint32_t t62 = t59 ^ t52;
  const uint32_t t63 = t60 ^ t51;
  const uint32_t t64 = t61 ^ t63;
  const uint32_t t65 = t53 ^ t62;
  const uint32_t t66 = t58 ^ t62;
  const uint32_t t67 = t51 ^ t52 ^ t53;
  const uint32_t t68 = t64;
  const uint32_t t69 = t52 ^ t54 ^ t64;
  const uint32_t t70 = t53 ^ t63;
  const uint32_t t71 = t65;
  const uint32_t t72 = t59 ^ t60;
  const uint32_t t73 = t54 ^ t65;
  x0 = t66;
  x1 = t67;
  x2 = t68;
  x3 = t69;
  x4 = t70;
  x5 = t71;
  x6 = t72;
  x7 = t73;
}

}  // namespace bs
}  // namespace aesgb
