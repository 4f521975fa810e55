"""GB300-native pseudopotential MRT lattice Boltzmann step with improved virtual-density contact
angles on curved walls (Li, Yu & Luo, arXiv:1908.04443).

The computation lives in liblbmwet.so (C ABI, include/lbmwet.h); `lbmwet` is its Python binding.
Import `paper_1908_04443_gb300.lbmwet` explicitly: importing the package itself loads nothing.
"""
