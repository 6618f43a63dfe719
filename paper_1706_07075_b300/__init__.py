"""List-mode TOF-MLEM (arXiv:1706.07075) on NVIDIA B300: the CUDA library
librecon.so behind include/recon.h and its thin Python binding.

    from paper_1706_07075_b300 import binding   # C-ABI, same names as recon.h
    from paper_1706_07075_b300 import synth     # seeded synthetic inputs
"""
