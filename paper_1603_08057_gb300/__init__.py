"""GB300-native recursive skeletonization factorization (RSF) for Gaussian
process log-likelihoods and scores on 2-D point sets.

The compute path is the C-ABI library built from ``csrc/`` (hand-written
CUDA for sm_103a); ``binding`` marshals arguments to it.  Importing this
package does not load the library; the first call does, and fails loudly if it
is missing.
"""
