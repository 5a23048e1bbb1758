// ddsg_tables.h -- host-side facts about a handle's uploaded grid tables that
// other translation units (the IRBC step) size their work by.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/ddsg.h"

namespace ddsg {
// Number of level tuples each component's evaluation walks in `form` (all of
// them in the paper form, those with every level >= 2 in the slice-free form);
// a point query activates at most one point per tuple. Needs uploaded tables
// (DDSG_ERR_STATE otherwise).
int handle_comp_tuples(hdmr_t *h, int form, std::vector<int32_t> &out);
}  // namespace ddsg
