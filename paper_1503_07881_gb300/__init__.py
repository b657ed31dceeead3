"""GB300-native table->graph conversion (Ringo, SIGMOD'15, Section 3.4).

The conversion runs in hand-written CUDA for sm_103a inside ``libringo.so``
(C ABI: include/ringo.h); :mod:`.ringo` is its thin Python binding.
"""
from .ringo import (RINGO_IN, RINGO_OUT, Graph, RingoError, load, ringo_profile_start,
                    ringo_profile_stop, ringo_table_to_graph, ringo_table_to_graph_host,
                    ringo_version)

__all__ = ["RINGO_IN", "RINGO_OUT", "Graph", "RingoError", "load", "ringo_profile_start",
           "ringo_profile_stop", "ringo_table_to_graph", "ringo_table_to_graph_host",
           "ringo_version"]
