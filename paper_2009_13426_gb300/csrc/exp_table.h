// Generated by gen_exp_table.py: constants of the table-driven FP64
// exponential (Tang's method), each computed with 60-digit decimal
// arithmetic and rounded to the nearest double.
#pragma once
namespace alb {
constexpr double EXPT_INV_L = 0x1.71547652b82fep+5;  // 32 / ln 2
constexpr double EXPT_L_HI = 0x1.62e42fefa0000p-6;   // ln2/32, 38 significant bits
constexpr double EXPT_L_LO = 0x1.cf79abc9e3b3ap-45;   // ln2/32 - EXPT_L_HI
constexpr double EXPT_C2 = 0x1.0000000000000p-1;  // 1/2!
constexpr double EXPT_C3 = 0x1.5555555555555p-3;  // 1/3!
constexpr double EXPT_C4 = 0x1.5555555555555p-5;  // 1/4!
constexpr double EXPT_C5 = 0x1.1111111111111p-7;  // 1/5!
constexpr double EXPT_C6 = 0x1.6c16c16c16c17p-10;  // 1/6!
}  // namespace alb
// T[j] = 2^(j/32), j = 0..31, as an initializer list
#define ALB_EXPT_TABLE_VALUES \
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, \
    0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0, \
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, \
    0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0, \
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, \
    0x1.3dea64c123422p+0, 0x1.44e086061892dp+0, \
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, \
    0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0, \
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, \
    0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0, \
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, \
    0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0, \
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, \
    0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0, \
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, \
    0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0
