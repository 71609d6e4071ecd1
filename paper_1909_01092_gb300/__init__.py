"""GB300-native fluctuating lattice Boltzmann step for a two-component
Shan-Chen mixture with a wetted finite-size particle (arXiv:1909.01092).

The compute path is the sm_103a CUDA library in `csrc/` behind the C-ABI of
`include/flbm.h`; `binding` is its thin ctypes wrapper.
"""
