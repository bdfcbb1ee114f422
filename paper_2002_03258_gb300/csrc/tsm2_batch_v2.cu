// Batch kernel, tile variant 2: stages 5, 4 rows per lane, 4 inner columns per warp.
#include "tsm2_batch_kernel.cuh"

namespace tsm2 {
namespace {

constexpr int kStages = 5;  // pipeline stages
constexpr int kNV = 1;      // 16-byte row vectors per lane (rows of C per lane = 4 kNV)
constexpr int kPregs = 56; // producer warpgroup registers per thread (consumers: the rest)
constexpr int kJW = 4;      // TSM2R: inner columns per warp and stage (8 warps split a stage)

// TSM2R schedule: 8 warps split the inner columns of a stage, partial sums
// meet in shared memory once per row block; B row-major for 16 columns.
template <int KC>
using VR = Cfg<float, KC, kNV, 1, 8, 1, kJW, kStages, false, 0, (KC >= 12)>;
// TSM2L schedule: warps split the rows (and for KC >= 16 the C columns),
// B resident (n <= 64), whole row blocks.
template <int KC>
using VW = Cfg<float, KC, kNV, (KC >= 16 ? 4 : 8), 1, (KC >= 16 ? 2 : 1), (KC >= 16 ? 2 : 1) * kJW, kStages, true, 64,
               ((KC / (KC >= 16 ? 2 : 1)) % 4 == 0)>;

const BatchClass kSlots[] = {
    class_of<VR<8>>('r', "v2_r_kc8"),   class_of<VR<12>>('r', "v2_r_kc12"), class_of<VR<16>>('r', "v2_r_kc16"),
    class_of<VW<8>>('w', "v2_l_kc8"),   class_of<VW<16>>('w', "v2_l_kc16"),
    class_of<VW<24>>('w', "v2_l_kc24"), class_of<VW<32>>('w', "v2_l_kc32"),
};

}  // namespace

const BatchMenu *batch_menu_v2() {
    static const BatchMenu menu = {
        "stages 5, 4 rows per lane, 4 inner columns per warp", kStages, 4 * kNV, kJW, 7,
        {&kSlots[0], &kSlots[1], &kSlots[2], &kSlots[3], &kSlots[4], &kSlots[5], &kSlots[6], nullptr},
        &launch_batch_kernel<kPregs, VR<8>, VR<12>, VR<16>, VW<8>, VW<16>, VW<24>, VW<32>>};
    return &menu;
}

}  // namespace tsm2
