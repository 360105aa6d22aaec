// Library-internal helpers shared by the C-ABI translation units.
#pragma once

// Records the diagnostic string returned by mlvs_last_error(NULL) for the calling thread.
void mlvs_internal_set_error(const char* msg);
