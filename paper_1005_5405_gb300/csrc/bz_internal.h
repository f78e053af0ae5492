// bz_internal.h -- helpers shared by the library's translation units.
#pragma once

// Stores the text returned by bz_last_error() on this thread.
void bz_record_error(const char *msg);
