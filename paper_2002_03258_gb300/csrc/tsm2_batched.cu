// Tile variants of the batch kernel (tsm2_batch_kernel.cuh) and their menus.
//
// Each variant is one kernel holding seven tile classes: TSM2R with 8, 12 or
// 16 C columns and TSM2L (whole row blocks, B resident) with 8, 16, 24 or 32.  A
// problem's column chunk goes to the narrowest class of its schedule that
// holds it (or, with the merge flags, to the widest).  The variants differ in
// the tile parameters the paper leaves to offline tuning (t1, t3 and tcf,
// Sec. 3.1.9 and 3.2.2): pipeline stages, rows of C per lane and inner
// columns per warp and stage.  The variants are compiled in separate
// translation units (tsm2_batch_v*.cu) so they build in parallel.
#include "internal.h"

namespace tsm2 {

const BatchMenu *batch_menu_v0();
const BatchMenu *batch_menu_v1();
const BatchMenu *batch_menu_v2();
const BatchMenu *batch_menu_v3();

int batch_menu_count() { return 4; }

const BatchMenu *batch_menu(int variant) {
    switch (variant) {
    case 0: return batch_menu_v0();
    case 1: return batch_menu_v1();
    case 2: return batch_menu_v2();
    case 3: return batch_menu_v3();
    default: return nullptr;
    }
}

}  // namespace tsm2
