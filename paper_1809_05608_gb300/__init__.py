"""GB300-native implicit MGFLD neutrino-transport step (CHIMERA, Bruenn et al.).

The compute path is the CUDA library ``libmgfld`` (C ABI, ``include/mgfld.h``);
``paper_1809_05608_gb300.mgfld`` is its thin Python binding and
``paper_1809_05608_gb300.problems`` manufactures seeded synthetic inputs.
"""
