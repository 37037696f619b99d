/*
 * onesweep_debug.h - test hooks of the GB300 Onesweep library. Not part of
 * the sort's interface: these change the behaviour of every later sort in
 * the process (they exist so tests can reach failure and large-problem
 * paths on small inputs), so product code does not include this header.
 * Declarations only; the library exports them.
 */
#ifndef ONESWEEP_DEBUG_H
#define ONESWEEP_DEBUG_H

#include "onesweep.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Fault injection for tests of the look-back wait limit (not part of the
 * method). With tile >= 0, every later binning pass skips all status-counter
 * publishes of that tile, so the tiles after it wait until `spin_limit`
 * polls have gone by, record OS_ERR_TIMEOUT and finish with invalid output.
 * tile = -1 switches injection off; spin_limit = 0 restores the default
 * limit. Process-wide setting (atomic), applied when a sort is planned.
 */
OS_API void os_debug_set_lookback_fault(int64_t tile, uint32_t spin_limit);

/*
 * Strip length of single-array sorts (Section 3, "Handling very large
 * problems"): a pass over more keys than one strip runs as one binning launch
 * per strip, each strip a chain of its own, the next strip's bins starting
 * where the previous strip's ended. Strips are at most 2^30 - 1 keys (every
 * look-back count stays below the 30-bit limit) and of equal length in whole
 * tiles; this sets that maximum, so tests can run the multi-strip path on
 * small inputs. `keys` is clamped to [2^16, 2^30 - 1]; 0 restores the
 * default. Returns the value set. Process-wide (atomic), applied when a sort is
 * planned; a workspace sized for n fits any strip length.
 */
OS_API uint64_t os_debug_set_strip_keys(uint64_t keys);

#ifdef __cplusplus
}
#endif

#endif /* ONESWEEP_DEBUG_H */
