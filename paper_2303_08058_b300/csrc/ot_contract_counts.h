// Generated by gen_contract.py -- do not edit.
// Operation counts of generated contractions (host and device).
#pragma once

// FP64 adds and FMAs of ot_mclass_fwd_z<Z>[_ang], indexed [ang][Z]
constexpr int OT_MCLASS_ADDS[2][7] = {{232, 70, 70, 16, 70, 16, 16}, {309, 95, 95, 22, 95, 22, 22}};
constexpr int OT_MCLASS_FMAS[2][7] = {{70, 40, 40, 22, 40, 22, 22}, {100, 56, 56, 31, 56, 31, 31}};
// FP64 adds of ot_mclass_fwd_x_z<Z>[_ang] (x stage prebuilt; 0 for Z with bit 0), [ang][Z]
constexpr int OT_MCLASS_X_ADDS[2][7] = {{132, 0, 30, 0, 30, 0, 0}, {181, 0, 41, 0, 41, 0, 0}};
// FP64 adds of ot_mclass_fwd_xy_z<Z>[_ang] (x and y stages prebuilt; 0 for Z with bit 0 or 1), [ang][Z]
constexpr int OT_MCLASS_XY_ADDS[2][7] = {{56, 0, 0, 0, 0, 0, 0}, {77, 0, 0, 0, 0, 0, 0}};
// FP64 adds of ot_mclass_adj_x_z<Z> (x stage prebuilt; 0 for Z with bit 0)
constexpr int OT_MCLASS_ADJ_X_ADDS[7] = {132, 0, 30, 0, 30, 0, 0};
// FP64 adds and FMAs of ot_mclass_adj_z<Z>
constexpr int OT_MCLASS_ADJ_ADDS[7] = {232, 70, 70, 16, 70, 16, 16};
constexpr int OT_MCLASS_ADJ_FMAS[7] = {70, 40, 40, 22, 40, 22, 22};
