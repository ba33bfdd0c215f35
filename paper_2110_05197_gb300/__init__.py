"""GB300-native two-component lattice Boltzmann step (colour-gradient and Shan-Chen models
of arXiv 2110.05197) behind a small C-ABI library.

The CUDA library is loaded on first use by :mod:`paper_2110_05197_gb300.lbm`; importing the
package itself loads nothing, so :mod:`paper_2110_05197_gb300.inputs` can be used on hosts
without a GPU.
"""
