// scan_ac_wide.cu -- the plain Aho-Corasick scan kernel (ac_scan_kernel.cuh)
// instantiated with a 768-thread launch bound, for plans of more than 16
// warps per CTA on ACGT tables: 24 warps hide more of the dependent
// shared-memory (or L2) latency of the walk, at up to 85 registers per
// thread. A translation unit of its own, so it compiles beside scan_ac.cu.
#include "ac_scan_kernel.cuh"

namespace pm {

const Variant kWideVariants[kWideGroups * 3] = {
    {ac_scan_kernel<uint16_t, 6, 1, true, false, false, false, 768>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, false, false, 768>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, false, false, 768>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, false, false, 768>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, false, false, 768>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, false, false, 768>, 2, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, true, false, 768>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, true, false, 768>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, true, false, 768>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, true, false, 768>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, true, false, 768>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, true, false, 768>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true, true, false, 768>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true, true, false, 768>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true, true, false, 768>, 4, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, false, true, 768>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, false, true, 768>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, false, true, 768>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, false, true, 768>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, false, true, 768>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, false, true, 768>, 2, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, true, true, 768>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, true, true, 768>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, true, true, 768>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, true, true, 768>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, true, true, 768>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, true, true, 768>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true, true, true, 768>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true, true, true, 768>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true, true, true, 768>, 4, 4, true, true},
};

}  // namespace pm
