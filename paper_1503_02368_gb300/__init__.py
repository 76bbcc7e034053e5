"""GB300 (sm_103a) pattern-count engine: generic worst-case optimal join
over a device-resident trie of uint/bitset neighbour sets (EmptyHeaded,
arXiv 1503.02368).  The Python layer only marshals arguments into the C ABI
of ``libeh.so`` (declared in ``include/eh.h``)."""
from .eh import (ORDERINGS, PATTERNS, EHError, Server, Trie, batch_profile, build_opts, exec_opts,  # noqa: F401
                 lib, library_path, range_bounds, trim_memory)
