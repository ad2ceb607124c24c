"""GB300-native AdamW-GS optimizer step (arXiv 2601.16736).

The CUDA library is loaded on first use of ``paper_2601_16736_gb300.gsopt``;
importing the package alone touches no GPU code.
"""
