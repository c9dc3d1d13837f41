// scan_ac_wide_counts.cu -- the 768-thread instances of the plain
// Aho-Corasick scan kernel (ac_scan_kernel.cuh) for counts-only scans: the
// walk records no step bits, one instruction less per text byte. Same order
// as kWideVariants; a translation unit of its own, so it compiles beside the
// others.
#include "ac_scan_kernel.cuh"

namespace pm {

const Variant kWideCountsVariants[kWideGroups * 3] = {
    {ac_scan_kernel<uint16_t, 6, 1, true, false, false, false, 768, true>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, false, false, 768, true>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, false, false, 768, true>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, false, false, 768, true>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, false, false, 768, true>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, false, false, 768, true>, 2, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, true, false, 768, true>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, true, false, 768, true>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, true, false, 768, true>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, true, false, 768, true>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, true, false, 768, true>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, true, false, 768, true>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true, true, false, 768, true>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true, true, false, 768, true>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true, true, false, 768, true>, 4, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, false, true, 768, true>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, false, true, 768, true>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, false, true, 768, true>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, false, true, 768, true>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, false, true, 768, true>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, false, true, 768, true>, 2, 4, true, true},
    {ac_scan_kernel<uint16_t, 6, 1, true, false, true, true, 768, true>, 2, 1, true, false},
    {ac_scan_kernel<uint16_t, 7, 2, true, false, true, true, 768, true>, 2, 2, true, false},
    {ac_scan_kernel<uint16_t, 9, 4, true, false, true, true, 768, true>, 2, 4, true, false},
    {ac_scan_kernel<uint16_t, 6, 1, true, true, true, true, 768, true>, 2, 1, true, true},
    {ac_scan_kernel<uint16_t, 7, 2, true, true, true, true, 768, true>, 2, 2, true, true},
    {ac_scan_kernel<uint16_t, 9, 4, true, true, true, true, 768, true>, 2, 4, true, true},
    {ac_scan_kernel<uint32_t, 6, 1, true, true, true, true, 768, true>, 4, 1, true, true},
    {ac_scan_kernel<uint32_t, 7, 2, true, true, true, true, 768, true>, 4, 2, true, true},
    {ac_scan_kernel<uint32_t, 9, 4, true, true, true, true, 768, true>, 4, 4, true, true},
};

}  // namespace pm
