"""GB300-native bi-directional pedestrian cellular automaton (LEM and ACO).

The compute path is the CUDA library ``libpedsim.so`` (sm_103a), reached through
the C ABI declared in ``include/pedsim.h``; ``pedsim`` is its thin Python
binding.  Importing this package does not load the library; importing
``paper_1412_4933_gb300.pedsim`` does, and fails loudly when it is missing.
"""
