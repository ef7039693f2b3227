/* Generated by paper_2002_05599_gb300/netgen/netgen.py -- do not edit.
 *
 * SN_NET_<n>(CE) expands to CE(i, j) for every comparator of the n-channel
 * sorting network in execution order: channels are 0-based, i < j, and the
 * comparator leaves the smaller value on channel i (Sec. 2.1).  Every
 * network was checked on all 2^n 0-1 inputs by the generator.
 */
#pragma once

/* n=2: 1 comparators, depth 1, from batcher-odd-even-top-top-top-top-top-top */
#define SN_NET_SIZE_2 1
#define SN_NET_2(CE) CE(0,1)

/* n=3: 3 comparators, depth 3, from batcher-odd-even-top-top-top-bottom-bottom */
#define SN_NET_SIZE_3 3
#define SN_NET_3(CE) CE(0,1) CE(0,2) CE(1,2)

/* n=4: 5 comparators, depth 3, from batcher-odd-even-top-top-bottom-bottom */
#define SN_NET_SIZE_4 5
#define SN_NET_4(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2)

/* n=5: 9 comparators, depth 5, from batcher-odd-even-top-top-top */
#define SN_NET_SIZE_5 9
#define SN_NET_5(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(0,4) CE(2,4) CE(1,2) CE(3,4)

/* n=6: 12 comparators, depth 6, from batcher-odd-even-top-top */
#define SN_NET_SIZE_6 12
#define SN_NET_6(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(4,5) CE(0,4) CE(2,4) CE(1,5) CE(3,5) CE(1,2) CE(3,4)

/* n=7: 16 comparators, depth 6, from batcher-odd-even-top */
#define SN_NET_SIZE_7 16
#define SN_NET_7(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(4,5) CE(4,6) CE(5,6) CE(0,4) CE(2,6) CE(2,4) CE(1,5) CE(3,5) CE(1,2) CE(3,4) CE(5,6)

/* n=8: 19 comparators, depth 6, from batcher-odd-even */
#define SN_NET_SIZE_8 19
#define SN_NET_8(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(4,5) CE(6,7) CE(4,6) CE(5,7) CE(5,6) CE(0,4) CE(2,6) CE(2,4) CE(1,5) CE(3,7) CE(3,5) CE(1,2) CE(3,4) CE(5,6)

/* n=9: 25 comparators, depth 8, from search(prefix=levels<=5 of the chosen n=12 network, restarts=2000, seed=1)-bottom-bottom-bottom */
#define SN_NET_SIZE_9 25
#define SN_NET_9(CE) CE(1,2) CE(3,4) CE(5,6) CE(7,8) CE(1,3) CE(5,7) CE(2,4) CE(6,8) CE(0,4) CE(0,8) CE(2,7) CE(3,6) CE(4,8) CE(1,5) CE(2,3) CE(6,7) CE(0,5) CE(5,6) CE(4,7) CE(3,5) CE(4,6) CE(0,2) CE(0,1) CE(4,5) CE(2,3)

/* n=10: 29 comparators, depth 9, from paper10 */
#define SN_NET_SIZE_10 29
#define SN_NET_10(CE) CE(4,9) CE(3,8) CE(2,7) CE(1,6) CE(0,5) CE(1,4) CE(6,9) CE(0,3) CE(5,8) CE(0,2) CE(3,6) CE(7,9) CE(0,1) CE(2,4) CE(5,7) CE(8,9) CE(1,2) CE(4,6) CE(7,8) CE(3,5) CE(2,5) CE(6,8) CE(1,3) CE(4,7) CE(2,3) CE(6,7) CE(3,4) CE(5,6) CE(4,5)

/* n=11: 35 comparators, depth 9, from search(prefix=levels<=5 of the chosen n=12 network, restarts=2000, seed=1)-top */
#define SN_NET_SIZE_11 35
#define SN_NET_11(CE) CE(0,1) CE(2,3) CE(4,5) CE(6,7) CE(8,9) CE(0,2) CE(4,6) CE(8,10) CE(1,3) CE(5,7) CE(0,4) CE(1,5) CE(2,6) CE(3,7) CE(0,8) CE(1,9) CE(2,10) CE(5,10) CE(6,9) CE(1,2) CE(4,8) CE(5,6) CE(9,10) CE(3,8) CE(2,3) CE(8,9) CE(1,4) CE(7,10) CE(6,8) CE(7,9) CE(3,5) CE(2,4) CE(3,4) CE(7,8) CE(5,6)

/* n=12: 39 comparators, depth 9, from search(prefix=levels<=5 of the chosen n=12 network, restarts=2000, seed=1) */
#define SN_NET_SIZE_12 39
#define SN_NET_12(CE) CE(0,1) CE(2,3) CE(4,5) CE(6,7) CE(8,9) CE(10,11) CE(0,2) CE(4,6) CE(8,10) CE(1,3) CE(5,7) CE(9,11) CE(0,4) CE(1,5) CE(2,6) CE(3,7) CE(0,8) CE(1,9) CE(2,10) CE(3,11) CE(5,10) CE(6,9) CE(7,11) CE(1,2) CE(4,8) CE(5,6) CE(9,10) CE(3,8) CE(2,3) CE(8,9) CE(1,4) CE(7,10) CE(6,8) CE(7,9) CE(3,5) CE(2,4) CE(3,4) CE(7,8) CE(5,6)

/* n=13: 45 comparators, depth 10, from evolve(n=13, target=45, seed=35, reflection, prefix=(0,1)(2,3)(4,5)(7,8)(9,10)(11,12), EVOLVE_RANDOM=40, EVOLVE_WORSE=20) */
#define SN_NET_SIZE_13 45
#define SN_NET_13(CE) CE(0,1) CE(2,3) CE(4,5) CE(7,8) CE(9,10) CE(11,12) CE(3,10) CE(2,9) CE(5,8) CE(0,11) CE(4,7) CE(1,12) CE(0,2) CE(1,5) CE(6,8) CE(10,12) CE(8,12) CE(6,10) CE(4,6) CE(0,4) CE(7,11) CE(2,6) CE(9,11) CE(1,9) CE(3,5) CE(5,8) CE(3,7) CE(2,4) CE(1,3) CE(6,9) CE(10,11) CE(5,10) CE(8,11) CE(5,7) CE(7,9) CE(1,2) CE(3,4) CE(5,6) CE(8,10) CE(8,9) CE(6,7) CE(2,3) CE(4,5) CE(5,6) CE(3,4)

/* n=14: 51 comparators, depth 10, from paper16-top-top */
#define SN_NET_SIZE_14 51
#define SN_NET_14(CE) CE(0,1) CE(2,3) CE(4,5) CE(6,7) CE(8,9) CE(10,11) CE(12,13) CE(0,2) CE(4,6) CE(8,10) CE(1,3) CE(5,7) CE(9,11) CE(0,4) CE(8,12) CE(1,5) CE(9,13) CE(2,6) CE(3,7) CE(0,8) CE(1,9) CE(2,10) CE(3,11) CE(4,12) CE(5,13) CE(5,10) CE(6,9) CE(3,12) CE(7,11) CE(1,2) CE(4,8) CE(1,4) CE(7,13) CE(2,8) CE(2,4) CE(5,6) CE(9,10) CE(11,13) CE(3,8) CE(7,12) CE(6,8) CE(10,12) CE(3,5) CE(7,9) CE(3,4) CE(5,6) CE(7,8) CE(9,10) CE(11,12) CE(6,7) CE(8,9)

/* n=15: 56 comparators, depth 10, from paper16-top */
#define SN_NET_SIZE_15 56
#define SN_NET_15(CE) CE(0,1) CE(2,3) CE(4,5) CE(6,7) CE(8,9) CE(10,11) CE(12,13) CE(0,2) CE(4,6) CE(8,10) CE(12,14) CE(1,3) CE(5,7) CE(9,11) CE(0,4) CE(8,12) CE(1,5) CE(9,13) CE(2,6) CE(10,14) CE(3,7) CE(0,8) CE(1,9) CE(2,10) CE(3,11) CE(4,12) CE(5,13) CE(6,14) CE(5,10) CE(6,9) CE(3,12) CE(13,14) CE(7,11) CE(1,2) CE(4,8) CE(1,4) CE(7,13) CE(2,8) CE(11,14) CE(2,4) CE(5,6) CE(9,10) CE(11,13) CE(3,8) CE(7,12) CE(6,8) CE(10,12) CE(3,5) CE(7,9) CE(3,4) CE(5,6) CE(7,8) CE(9,10) CE(11,12) CE(6,7) CE(8,9)

/* n=16: 60 comparators, depth 10, from paper16 */
#define SN_NET_SIZE_16 60
#define SN_NET_16(CE) CE(0,1) CE(2,3) CE(4,5) CE(6,7) CE(8,9) CE(10,11) CE(12,13) CE(14,15) CE(0,2) CE(4,6) CE(8,10) CE(12,14) CE(1,3) CE(5,7) CE(9,11) CE(13,15) CE(0,4) CE(8,12) CE(1,5) CE(9,13) CE(2,6) CE(10,14) CE(3,7) CE(11,15) CE(0,8) CE(1,9) CE(2,10) CE(3,11) CE(4,12) CE(5,13) CE(6,14) CE(7,15) CE(5,10) CE(6,9) CE(3,12) CE(13,14) CE(7,11) CE(1,2) CE(4,8) CE(1,4) CE(7,13) CE(2,8) CE(11,14) CE(2,4) CE(5,6) CE(9,10) CE(11,13) CE(3,8) CE(7,12) CE(6,8) CE(10,12) CE(3,5) CE(7,9) CE(3,4) CE(5,6) CE(7,8) CE(9,10) CE(11,12) CE(6,7) CE(8,9)

/* Bose-Nelson networks (recursive construction, emission order of the
 * recursion): SN_BN_<n>(CE), same conventions as SN_NET_<n>. */
/* n=2: 1 comparators, depth 1 */
#define SN_BN_SIZE_2 1
#define SN_BN_2(CE) CE(0,1)
/* n=3: 3 comparators, depth 3 */
#define SN_BN_SIZE_3 3
#define SN_BN_3(CE) CE(1,2) CE(0,2) CE(0,1)
/* n=4: 5 comparators, depth 3 */
#define SN_BN_SIZE_4 5
#define SN_BN_4(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2)
/* n=5: 9 comparators, depth 6 */
#define SN_BN_SIZE_5 9
#define SN_BN_5(CE) CE(0,1) CE(3,4) CE(2,4) CE(2,3) CE(0,3) CE(0,2) CE(1,4) CE(1,3) CE(1,2)
/* n=6: 12 comparators, depth 6 */
#define SN_BN_SIZE_6 12
#define SN_BN_6(CE) CE(1,2) CE(0,2) CE(0,1) CE(4,5) CE(3,5) CE(3,4) CE(0,3) CE(1,4) CE(2,5) CE(2,4) CE(1,3) CE(2,3)
/* n=7: 16 comparators, depth 7 */
#define SN_BN_SIZE_7 16
#define SN_BN_7(CE) CE(1,2) CE(0,2) CE(0,1) CE(3,4) CE(5,6) CE(3,5) CE(4,6) CE(4,5) CE(0,4) CE(0,3) CE(1,5) CE(2,6) CE(2,5) CE(1,3) CE(2,4) CE(2,3)
/* n=8: 19 comparators, depth 7 */
#define SN_BN_SIZE_8 19
#define SN_BN_8(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(4,5) CE(6,7) CE(4,6) CE(5,7) CE(5,6) CE(0,4) CE(1,5) CE(1,4) CE(2,6) CE(3,7) CE(3,6) CE(2,4) CE(3,5) CE(3,4)
/* n=9: 27 comparators, depth 11 */
#define SN_BN_SIZE_9 27
#define SN_BN_9(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(4,5) CE(7,8) CE(6,8) CE(6,7) CE(4,7) CE(4,6) CE(5,8) CE(5,7) CE(5,6) CE(0,5) CE(0,4) CE(1,6) CE(1,5) CE(1,4) CE(2,7) CE(3,8) CE(3,7) CE(2,5) CE(2,4) CE(3,6) CE(3,5) CE(3,4)
/* n=10: 32 comparators, depth 11 */
#define SN_BN_SIZE_10 32
#define SN_BN_10(CE) CE(0,1) CE(3,4) CE(2,4) CE(2,3) CE(0,3) CE(0,2) CE(1,4) CE(1,3) CE(1,2) CE(5,6) CE(8,9) CE(7,9) CE(7,8) CE(5,8) CE(5,7) CE(6,9) CE(6,8) CE(6,7) CE(0,5) CE(1,6) CE(1,5) CE(2,7) CE(3,8) CE(4,9) CE(4,8) CE(3,7) CE(4,7) CE(2,5) CE(3,6) CE(4,6) CE(3,5) CE(4,5)
/* n=11: 38 comparators, depth 12 */
#define SN_BN_SIZE_11 38
#define SN_BN_11(CE) CE(0,1) CE(3,4) CE(2,4) CE(2,3) CE(0,3) CE(0,2) CE(1,4) CE(1,3) CE(1,2) CE(6,7) CE(5,7) CE(5,6) CE(9,10) CE(8,10) CE(8,9) CE(5,8) CE(6,9) CE(7,10) CE(7,9) CE(6,8) CE(7,8) CE(0,6) CE(0,5) CE(1,7) CE(1,6) CE(1,5) CE(2,8) CE(3,9) CE(4,10) CE(4,9) CE(3,8) CE(4,8) CE(2,5) CE(3,6) CE(4,7) CE(4,6) CE(3,5) CE(4,5)
/* n=12: 42 comparators, depth 12 */
#define SN_BN_SIZE_12 42
#define SN_BN_12(CE) CE(1,2) CE(0,2) CE(0,1) CE(4,5) CE(3,5) CE(3,4) CE(0,3) CE(1,4) CE(2,5) CE(2,4) CE(1,3) CE(2,3) CE(7,8) CE(6,8) CE(6,7) CE(10,11) CE(9,11) CE(9,10) CE(6,9) CE(7,10) CE(8,11) CE(8,10) CE(7,9) CE(8,9) CE(0,6) CE(1,7) CE(2,8) CE(2,7) CE(1,6) CE(2,6) CE(3,9) CE(4,10) CE(5,11) CE(5,10) CE(4,9) CE(5,9) CE(3,6) CE(4,7) CE(5,8) CE(5,7) CE(4,6) CE(5,6)
/* n=13: 50 comparators, depth 14 */
#define SN_BN_SIZE_13 50
#define SN_BN_13(CE) CE(1,2) CE(0,2) CE(0,1) CE(4,5) CE(3,5) CE(3,4) CE(0,3) CE(1,4) CE(2,5) CE(2,4) CE(1,3) CE(2,3) CE(7,8) CE(6,8) CE(6,7) CE(9,10) CE(11,12) CE(9,11) CE(10,12) CE(10,11) CE(6,10) CE(6,9) CE(7,11) CE(8,12) CE(8,11) CE(7,9) CE(8,10) CE(8,9) CE(0,7) CE(0,6) CE(1,8) CE(2,9) CE(2,8) CE(1,6) CE(2,7) CE(2,6) CE(3,10) CE(4,11) CE(5,12) CE(5,11) CE(4,10) CE(5,10) CE(3,7) CE(3,6) CE(4,8) CE(5,9) CE(5,8) CE(4,6) CE(5,7) CE(5,6)
/* n=14: 55 comparators, depth 14 */
#define SN_BN_SIZE_14 55
#define SN_BN_14(CE) CE(1,2) CE(0,2) CE(0,1) CE(3,4) CE(5,6) CE(3,5) CE(4,6) CE(4,5) CE(0,4) CE(0,3) CE(1,5) CE(2,6) CE(2,5) CE(1,3) CE(2,4) CE(2,3) CE(8,9) CE(7,9) CE(7,8) CE(10,11) CE(12,13) CE(10,12) CE(11,13) CE(11,12) CE(7,11) CE(7,10) CE(8,12) CE(9,13) CE(9,12) CE(8,10) CE(9,11) CE(9,10) CE(0,7) CE(1,8) CE(2,9) CE(2,8) CE(1,7) CE(2,7) CE(3,10) CE(4,11) CE(4,10) CE(5,12) CE(6,13) CE(6,12) CE(5,10) CE(6,11) CE(6,10) CE(3,7) CE(4,8) CE(4,7) CE(5,9) CE(6,9) CE(5,7) CE(6,8) CE(6,7)
/* n=15: 61 comparators, depth 15 */
#define SN_BN_SIZE_15 61
#define SN_BN_15(CE) CE(1,2) CE(0,2) CE(0,1) CE(3,4) CE(5,6) CE(3,5) CE(4,6) CE(4,5) CE(0,4) CE(0,3) CE(1,5) CE(2,6) CE(2,5) CE(1,3) CE(2,4) CE(2,3) CE(7,8) CE(9,10) CE(7,9) CE(8,10) CE(8,9) CE(11,12) CE(13,14) CE(11,13) CE(12,14) CE(12,13) CE(7,11) CE(8,12) CE(8,11) CE(9,13) CE(10,14) CE(10,13) CE(9,11) CE(10,12) CE(10,11) CE(0,8) CE(0,7) CE(1,9) CE(2,10) CE(2,9) CE(1,7) CE(2,8) CE(2,7) CE(3,11) CE(4,12) CE(4,11) CE(5,13) CE(6,14) CE(6,13) CE(5,11) CE(6,12) CE(6,11) CE(3,7) CE(4,8) CE(4,7) CE(5,9) CE(6,10) CE(6,9) CE(5,7) CE(6,8) CE(6,7)
/* n=16: 65 comparators, depth 15 */
#define SN_BN_SIZE_16 65
#define SN_BN_16(CE) CE(0,1) CE(2,3) CE(0,2) CE(1,3) CE(1,2) CE(4,5) CE(6,7) CE(4,6) CE(5,7) CE(5,6) CE(0,4) CE(1,5) CE(1,4) CE(2,6) CE(3,7) CE(3,6) CE(2,4) CE(3,5) CE(3,4) CE(8,9) CE(10,11) CE(8,10) CE(9,11) CE(9,10) CE(12,13) CE(14,15) CE(12,14) CE(13,15) CE(13,14) CE(8,12) CE(9,13) CE(9,12) CE(10,14) CE(11,15) CE(11,14) CE(10,12) CE(11,13) CE(11,12) CE(0,8) CE(1,9) CE(1,8) CE(2,10) CE(3,11) CE(3,10) CE(2,8) CE(3,9) CE(3,8) CE(4,12) CE(5,13) CE(5,12) CE(6,14) CE(7,15) CE(7,14) CE(6,12) CE(7,13) CE(7,12) CE(4,8) CE(5,9) CE(5,8) CE(6,10) CE(7,11) CE(7,10) CE(6,8) CE(7,9) CE(7,8)

/* 32-lane warp network (17..32 items): lane l exchanges with lane l ^ M at
 * each step M below; the lower lane keeps the smaller item. */
#define SN_WARP32_STEPS 15
#define SN_WARP32_SCHEDULE(STEP) STEP(1) STEP(3) STEP(1) STEP(7) STEP(2) STEP(1) STEP(15) STEP(4) STEP(2) STEP(1) STEP(31) STEP(8) STEP(4) STEP(2) STEP(1)
