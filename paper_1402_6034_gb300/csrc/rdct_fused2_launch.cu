// Launches of the fused kernel: one specialisation per r (instantiated in
// rdct_fused2_r*.cu), for a single plane or for one r group of a batch.
#include <algorithm>

#include "rdct_fused2.cuh"

namespace rdct {

extern template cudaError_t launch_fused2_r<1>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<2>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<3>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<4>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<5>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<6>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<7>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<8>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<9>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<10>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<11>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<12>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<13>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<14>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<15>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<16>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<17>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<18>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<19>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<20>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<21>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<22>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<23>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<24>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<25>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<26>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<27>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<28>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<29>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<30>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<31>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<32>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<33>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<34>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<35>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<36>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<37>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<38>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<39>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<40>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<41>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<42>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<43>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<44>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<45>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<46>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<47>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<48>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<49>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<50>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<51>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<52>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<53>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<54>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<55>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<56>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<57>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<58>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<59>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<60>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<61>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<62>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<63>(const Fused2Args &, bool, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_r<64>(const Fused2Args &, bool, int, bool, cudaStream_t);

extern template cudaError_t launch_fused2_tma_r<1>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<2>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<3>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<4>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<5>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<6>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<7>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<8>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<9>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<10>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<11>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<12>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<13>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<14>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<15>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<16>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<17>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<18>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<19>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<20>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<21>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<22>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<23>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<24>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<25>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<26>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<27>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<28>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<29>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<30>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<31>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<32>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<33>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<34>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<35>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<36>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<37>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<38>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<39>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<40>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<41>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<42>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<43>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<44>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<45>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<46>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<47>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<48>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<49>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<50>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<51>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<52>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<53>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<54>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<55>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<56>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<57>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<58>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<59>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<60>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<61>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<62>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<63>(const TmaArgs &, int, bool, cudaStream_t);
extern template cudaError_t launch_fused2_tma_r<64>(const TmaArgs &, int, bool, cudaStream_t);

namespace {

cudaError_t launch_fused2_any(int r, const Fused2Args &a, bool single, int ctas_per_sm, bool overlap,
                              cudaStream_t s) {
    switch (r) {
        case 1: return launch_fused2_r<1>(a, single, ctas_per_sm, overlap, s);
        case 2: return launch_fused2_r<2>(a, single, ctas_per_sm, overlap, s);
        case 3: return launch_fused2_r<3>(a, single, ctas_per_sm, overlap, s);
        case 4: return launch_fused2_r<4>(a, single, ctas_per_sm, overlap, s);
        case 5: return launch_fused2_r<5>(a, single, ctas_per_sm, overlap, s);
        case 6: return launch_fused2_r<6>(a, single, ctas_per_sm, overlap, s);
        case 7: return launch_fused2_r<7>(a, single, ctas_per_sm, overlap, s);
        case 8: return launch_fused2_r<8>(a, single, ctas_per_sm, overlap, s);
        case 9: return launch_fused2_r<9>(a, single, ctas_per_sm, overlap, s);
        case 10: return launch_fused2_r<10>(a, single, ctas_per_sm, overlap, s);
        case 11: return launch_fused2_r<11>(a, single, ctas_per_sm, overlap, s);
        case 12: return launch_fused2_r<12>(a, single, ctas_per_sm, overlap, s);
        case 13: return launch_fused2_r<13>(a, single, ctas_per_sm, overlap, s);
        case 14: return launch_fused2_r<14>(a, single, ctas_per_sm, overlap, s);
        case 15: return launch_fused2_r<15>(a, single, ctas_per_sm, overlap, s);
        case 16: return launch_fused2_r<16>(a, single, ctas_per_sm, overlap, s);
        case 17: return launch_fused2_r<17>(a, single, ctas_per_sm, overlap, s);
        case 18: return launch_fused2_r<18>(a, single, ctas_per_sm, overlap, s);
        case 19: return launch_fused2_r<19>(a, single, ctas_per_sm, overlap, s);
        case 20: return launch_fused2_r<20>(a, single, ctas_per_sm, overlap, s);
        case 21: return launch_fused2_r<21>(a, single, ctas_per_sm, overlap, s);
        case 22: return launch_fused2_r<22>(a, single, ctas_per_sm, overlap, s);
        case 23: return launch_fused2_r<23>(a, single, ctas_per_sm, overlap, s);
        case 24: return launch_fused2_r<24>(a, single, ctas_per_sm, overlap, s);
        case 25: return launch_fused2_r<25>(a, single, ctas_per_sm, overlap, s);
        case 26: return launch_fused2_r<26>(a, single, ctas_per_sm, overlap, s);
        case 27: return launch_fused2_r<27>(a, single, ctas_per_sm, overlap, s);
        case 28: return launch_fused2_r<28>(a, single, ctas_per_sm, overlap, s);
        case 29: return launch_fused2_r<29>(a, single, ctas_per_sm, overlap, s);
        case 30: return launch_fused2_r<30>(a, single, ctas_per_sm, overlap, s);
        case 31: return launch_fused2_r<31>(a, single, ctas_per_sm, overlap, s);
        case 32: return launch_fused2_r<32>(a, single, ctas_per_sm, overlap, s);
        case 33: return launch_fused2_r<33>(a, single, ctas_per_sm, overlap, s);
        case 34: return launch_fused2_r<34>(a, single, ctas_per_sm, overlap, s);
        case 35: return launch_fused2_r<35>(a, single, ctas_per_sm, overlap, s);
        case 36: return launch_fused2_r<36>(a, single, ctas_per_sm, overlap, s);
        case 37: return launch_fused2_r<37>(a, single, ctas_per_sm, overlap, s);
        case 38: return launch_fused2_r<38>(a, single, ctas_per_sm, overlap, s);
        case 39: return launch_fused2_r<39>(a, single, ctas_per_sm, overlap, s);
        case 40: return launch_fused2_r<40>(a, single, ctas_per_sm, overlap, s);
        case 41: return launch_fused2_r<41>(a, single, ctas_per_sm, overlap, s);
        case 42: return launch_fused2_r<42>(a, single, ctas_per_sm, overlap, s);
        case 43: return launch_fused2_r<43>(a, single, ctas_per_sm, overlap, s);
        case 44: return launch_fused2_r<44>(a, single, ctas_per_sm, overlap, s);
        case 45: return launch_fused2_r<45>(a, single, ctas_per_sm, overlap, s);
        case 46: return launch_fused2_r<46>(a, single, ctas_per_sm, overlap, s);
        case 47: return launch_fused2_r<47>(a, single, ctas_per_sm, overlap, s);
        case 48: return launch_fused2_r<48>(a, single, ctas_per_sm, overlap, s);
        case 49: return launch_fused2_r<49>(a, single, ctas_per_sm, overlap, s);
        case 50: return launch_fused2_r<50>(a, single, ctas_per_sm, overlap, s);
        case 51: return launch_fused2_r<51>(a, single, ctas_per_sm, overlap, s);
        case 52: return launch_fused2_r<52>(a, single, ctas_per_sm, overlap, s);
        case 53: return launch_fused2_r<53>(a, single, ctas_per_sm, overlap, s);
        case 54: return launch_fused2_r<54>(a, single, ctas_per_sm, overlap, s);
        case 55: return launch_fused2_r<55>(a, single, ctas_per_sm, overlap, s);
        case 56: return launch_fused2_r<56>(a, single, ctas_per_sm, overlap, s);
        case 57: return launch_fused2_r<57>(a, single, ctas_per_sm, overlap, s);
        case 58: return launch_fused2_r<58>(a, single, ctas_per_sm, overlap, s);
        case 59: return launch_fused2_r<59>(a, single, ctas_per_sm, overlap, s);
        case 60: return launch_fused2_r<60>(a, single, ctas_per_sm, overlap, s);
        case 61: return launch_fused2_r<61>(a, single, ctas_per_sm, overlap, s);
        case 62: return launch_fused2_r<62>(a, single, ctas_per_sm, overlap, s);
        case 63: return launch_fused2_r<63>(a, single, ctas_per_sm, overlap, s);
        case 64: return launch_fused2_r<64>(a, single, ctas_per_sm, overlap, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused2_tma_any(int r, const TmaArgs &a, int ctas_per_sm, bool overlap, cudaStream_t s) {
    switch (r) {
        case 1: return launch_fused2_tma_r<1>(a, ctas_per_sm, overlap, s);
        case 2: return launch_fused2_tma_r<2>(a, ctas_per_sm, overlap, s);
        case 3: return launch_fused2_tma_r<3>(a, ctas_per_sm, overlap, s);
        case 4: return launch_fused2_tma_r<4>(a, ctas_per_sm, overlap, s);
        case 5: return launch_fused2_tma_r<5>(a, ctas_per_sm, overlap, s);
        case 6: return launch_fused2_tma_r<6>(a, ctas_per_sm, overlap, s);
        case 7: return launch_fused2_tma_r<7>(a, ctas_per_sm, overlap, s);
        case 8: return launch_fused2_tma_r<8>(a, ctas_per_sm, overlap, s);
        case 9: return launch_fused2_tma_r<9>(a, ctas_per_sm, overlap, s);
        case 10: return launch_fused2_tma_r<10>(a, ctas_per_sm, overlap, s);
        case 11: return launch_fused2_tma_r<11>(a, ctas_per_sm, overlap, s);
        case 12: return launch_fused2_tma_r<12>(a, ctas_per_sm, overlap, s);
        case 13: return launch_fused2_tma_r<13>(a, ctas_per_sm, overlap, s);
        case 14: return launch_fused2_tma_r<14>(a, ctas_per_sm, overlap, s);
        case 15: return launch_fused2_tma_r<15>(a, ctas_per_sm, overlap, s);
        case 16: return launch_fused2_tma_r<16>(a, ctas_per_sm, overlap, s);
        case 17: return launch_fused2_tma_r<17>(a, ctas_per_sm, overlap, s);
        case 18: return launch_fused2_tma_r<18>(a, ctas_per_sm, overlap, s);
        case 19: return launch_fused2_tma_r<19>(a, ctas_per_sm, overlap, s);
        case 20: return launch_fused2_tma_r<20>(a, ctas_per_sm, overlap, s);
        case 21: return launch_fused2_tma_r<21>(a, ctas_per_sm, overlap, s);
        case 22: return launch_fused2_tma_r<22>(a, ctas_per_sm, overlap, s);
        case 23: return launch_fused2_tma_r<23>(a, ctas_per_sm, overlap, s);
        case 24: return launch_fused2_tma_r<24>(a, ctas_per_sm, overlap, s);
        case 25: return launch_fused2_tma_r<25>(a, ctas_per_sm, overlap, s);
        case 26: return launch_fused2_tma_r<26>(a, ctas_per_sm, overlap, s);
        case 27: return launch_fused2_tma_r<27>(a, ctas_per_sm, overlap, s);
        case 28: return launch_fused2_tma_r<28>(a, ctas_per_sm, overlap, s);
        case 29: return launch_fused2_tma_r<29>(a, ctas_per_sm, overlap, s);
        case 30: return launch_fused2_tma_r<30>(a, ctas_per_sm, overlap, s);
        case 31: return launch_fused2_tma_r<31>(a, ctas_per_sm, overlap, s);
        case 32: return launch_fused2_tma_r<32>(a, ctas_per_sm, overlap, s);
        case 33: return launch_fused2_tma_r<33>(a, ctas_per_sm, overlap, s);
        case 34: return launch_fused2_tma_r<34>(a, ctas_per_sm, overlap, s);
        case 35: return launch_fused2_tma_r<35>(a, ctas_per_sm, overlap, s);
        case 36: return launch_fused2_tma_r<36>(a, ctas_per_sm, overlap, s);
        case 37: return launch_fused2_tma_r<37>(a, ctas_per_sm, overlap, s);
        case 38: return launch_fused2_tma_r<38>(a, ctas_per_sm, overlap, s);
        case 39: return launch_fused2_tma_r<39>(a, ctas_per_sm, overlap, s);
        case 40: return launch_fused2_tma_r<40>(a, ctas_per_sm, overlap, s);
        case 41: return launch_fused2_tma_r<41>(a, ctas_per_sm, overlap, s);
        case 42: return launch_fused2_tma_r<42>(a, ctas_per_sm, overlap, s);
        case 43: return launch_fused2_tma_r<43>(a, ctas_per_sm, overlap, s);
        case 44: return launch_fused2_tma_r<44>(a, ctas_per_sm, overlap, s);
        case 45: return launch_fused2_tma_r<45>(a, ctas_per_sm, overlap, s);
        case 46: return launch_fused2_tma_r<46>(a, ctas_per_sm, overlap, s);
        case 47: return launch_fused2_tma_r<47>(a, ctas_per_sm, overlap, s);
        case 48: return launch_fused2_tma_r<48>(a, ctas_per_sm, overlap, s);
        case 49: return launch_fused2_tma_r<49>(a, ctas_per_sm, overlap, s);
        case 50: return launch_fused2_tma_r<50>(a, ctas_per_sm, overlap, s);
        case 51: return launch_fused2_tma_r<51>(a, ctas_per_sm, overlap, s);
        case 52: return launch_fused2_tma_r<52>(a, ctas_per_sm, overlap, s);
        case 53: return launch_fused2_tma_r<53>(a, ctas_per_sm, overlap, s);
        case 54: return launch_fused2_tma_r<54>(a, ctas_per_sm, overlap, s);
        case 55: return launch_fused2_tma_r<55>(a, ctas_per_sm, overlap, s);
        case 56: return launch_fused2_tma_r<56>(a, ctas_per_sm, overlap, s);
        case 57: return launch_fused2_tma_r<57>(a, ctas_per_sm, overlap, s);
        case 58: return launch_fused2_tma_r<58>(a, ctas_per_sm, overlap, s);
        case 59: return launch_fused2_tma_r<59>(a, ctas_per_sm, overlap, s);
        case 60: return launch_fused2_tma_r<60>(a, ctas_per_sm, overlap, s);
        case 61: return launch_fused2_tma_r<61>(a, ctas_per_sm, overlap, s);
        case 62: return launch_fused2_tma_r<62>(a, ctas_per_sm, overlap, s);
        case 63: return launch_fused2_tma_r<63>(a, ctas_per_sm, overlap, s);
        case 64: return launch_fused2_tma_r<64>(a, ctas_per_sm, overlap, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fused2_tma_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks,
                                    const unsigned char *maps, unsigned long long *acc, unsigned long long *acc8,
                                    int r, int ctas_per_sm, bool overlap, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    TmaArgs a{};
    a.jobs = jobs;
    a.chunks = chunks;
    a.maps = maps;
    a.nchunks = nchunks;
    a.acc = acc;
    a.acc8 = acc8;
    return launch_fused2_tma_any(r, a, ctas_per_sm, overlap, s);
}

cudaError_t launch_fused2_single(const JobDesc &job, unsigned long long *acc, unsigned long long *acc8,
                                 int ctas_per_sm, int chunk_items, cudaStream_t s) {
    Fused2Args a{};
    a.single = job;
    const int64_t items = fused_items_of(job);
    if (chunk_items <= 0) {  // enough chunks for every resident warp, at most 16 strips each
        const int64_t warps = (int64_t)sm_count() * 16;
        chunk_items = (int)std::min<int64_t>(16, std::max<int64_t>(1, items / warps));
    }
    a.chunk_items = chunk_items;
    a.nchunks = (int32_t)((items + a.chunk_items - 1) / a.chunk_items);
    a.acc = acc;
    a.acc8 = acc8;
    if (a.nchunks == 0) return cudaSuccess;
    return launch_fused2_any(job.r, a, true, ctas_per_sm, false, s);
}

cudaError_t launch_fused2_batch(const JobDesc *jobs, const Chunk *chunks, int32_t nchunks, unsigned long long *acc,
                                unsigned long long *acc8, int r, int ctas_per_sm, bool overlap, cudaStream_t s) {
    if (nchunks <= 0) return cudaSuccess;
    Fused2Args a{};
    a.jobs = jobs;
    a.chunks = chunks;
    a.nchunks = nchunks;
    a.acc = acc;
    a.acc8 = acc8;
    return launch_fused2_any(r, a, false, ctas_per_sm, overlap, s);
}

}  // namespace rdct
